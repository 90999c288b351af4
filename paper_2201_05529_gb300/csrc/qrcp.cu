// QR-preconditioned one-sided Jacobi for the bond SVD (App. A.2 (f-g)).
//
// A one-sided Jacobi on a rank-deficient, strongly graded D needs many sweeps (26-32 on the
// five-site chain's 256x256 blocks); after a column-pivoted QR, D P = Q R, the same Jacobi on R^H
// converges in ~9 (Drmac and Veselic's preconditioning). Here:
//   1. k_qrcp: Householder QR with column pivoting of a copy of D, one thread-block cluster per
//      matrix (column swaps and trailing updates spread over its CTAs, cluster barriers between
//      the steps; exact trailing column norms recomputed at every step for the pivot choice);
//   2. k_qrcp_rh: B = R^H (lower triangular, Na x Na);
//   3. the grid Jacobi on B gives B = U' S V'^H, i.e. R = V' S U'^H and D = (Q V') S (P U')^H;
//   4. k_qrcp_vd: V_D = P U' (rows permuted back);
//   5. U_D = D V_D S^{-1} by an FP64 GEMM (k_mix_gemm op 2) and a column scaling. Its error in
//      column c is ~eps ||D|| / s_c, and that column enters the truncated state scaled by s_c, so
//      the state error stays at rounding level; Q is never formed.
#include <cooperative_groups.h>

#include "grid_sync.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace ptk {

namespace {

__device__ __forceinline__ void shape(const BondWork& W, int* Ma, int* Na) {
  const int mD = W.info[0], nD = W.info[1];
  const bool tr = W.info[2] != 0;
  *Ma = (mD > 0 && nD > 0) ? (tr ? nD : mD) : 0;
  *Na = (mD > 0 && nD > 0) ? (tr ? mD : nD) : 0;
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// two lane sums at once: lane 0 ends with the total of a, lane 16 with that of b
__device__ __forceinline__ double wsum2(double a, double b, int lane) {
  const bool hi = (lane & 16) != 0;
  double keep = hi ? b : a;
  keep += __shfl_xor_sync(0xffffffffu, hi ? a : b, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
  return keep;
}

}  // namespace

// Column-pivoted Householder QR in place on X (Ma x Na col-major, Ma >= Na); X's upper triangle
// becomes R; qperm[k] = original column of position k; nrm: Na doubles of scratch.
__global__ void __launch_bounds__(1024) k_qrcp(const BondWork* work, int n_work) {
  cg::cluster_group cl = cg::this_cluster();
  const int w = blockIdx.x / cl.num_blocks();
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  shape(W, &Ma, &Na);
  if (Na <= 0) return;
  double2* X = W.Y64;
  double* nrm = W.aux;
  int* qperm = W.qperm;
  const int rank = (int)cl.block_rank(), ncta = (int)cl.num_blocks();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwb = blockDim.x >> 5;
  const int gw = wid * ncta + rank, ngw = ncta * nwb;
  const int gt = rank * blockDim.x + tid, ngt = ncta * blockDim.x;
  __shared__ double s_red[32];
  __shared__ int s_piv;
  // copy D into the workspace, initial column norms, identity permutation
  for (size_t i = gt; i < (size_t)Ma * Na; i += ngt) X[i] = W.A[i];
  for (int k = gt; k < Na; k += ngt) __stcg(qperm + k, k);
  cl.sync();
  for (int k = gw; k < Na; k += ngw) {
    double s = 0;
    for (int r = lane; r < Ma; r += 32) {
      const double2 x = __ldcg(X + (size_t)k * Ma + r);
      s += x.x * x.x + x.y * x.y;
    }
    s = wsum(s);
    if (lane == 0) __stcg(nrm + k, s);
  }
  cl.sync();
  for (int j = 0; j < Na && j < Ma; ++j) {
    // pivot: the remaining column of largest norm (every CTA scans the same values in the same order)
    if (wid == 0) {
      double best = -1.0;
      int bi = j;
      for (int k = j + lane; k < Na; k += 32) {
        const double v = __ldcg(nrm + k);
        if (v > best || (v == best && k < bi)) { best = v; bi = k; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) s_piv = bi;
    }
    __syncthreads();
    const int p = s_piv;
    if (p != j) {
      double2* cj = X + (size_t)j * Ma;
      double2* cp = X + (size_t)p * Ma;
      for (int r = gt; r < Ma; r += ngt) {
        const double2 a = __ldcg(cj + r), b = __ldcg(cp + r);
        __stcg(cj + r, b);
        __stcg(cp + r, a);
      }
      cl.sync();                                  // all reads of the old columns done
      if (gt == 0) {
        const double t = __ldcg(nrm + j);
        __stcg(nrm + j, __ldcg(nrm + p));
        __stcg(nrm + p, t);
        const int q = __ldcg(qperm + j);
        __stcg(qperm + j, __ldcg(qperm + p));
        __stcg(qperm + p, q);
      }
    }
    cl.sync();
    // Householder vector of column j (rows j..Ma-1): every CTA computes the same scalars
    const double2* x = X + (size_t)j * Ma;
    double part = 0;
    for (int r = j + tid; r < Ma; r += blockDim.x) {
      const double2 v = __ldcg(x + r);
      part += v.x * v.x + v.y * v.y;
    }
    part = wsum(part);
    if (lane == 0) s_red[wid] = part;
    __syncthreads();
    if (wid == 0) {
      double t = lane < nwb ? s_red[lane] : 0.0;
      t = wsum(t);
      if (lane == 0) s_red[0] = t;
    }
    __syncthreads();
    const double nrm2 = s_red[0];
    __syncthreads();
    const double2 alpha = __ldcg(x + j);
    const double aabs = sqrt(alpha.x * alpha.x + alpha.y * alpha.y), xn = sqrt(nrm2);
    double tau = 0.0;
    double2 ph = make_double2(1.0, 0.0), beta = alpha, ujinv = make_double2(0.0, 0.0);
    if (xn > 0.0) {
      if (aabs > 0.0) ph = make_double2(alpha.x / aabs, alpha.y / aabs);
      beta = make_double2(-ph.x * xn, -ph.y * xn);
      const double2 uj = make_double2(ph.x * (aabs + xn), ph.y * (aabs + xn));   // alpha - beta
      const double uj2 = uj.x * uj.x + uj.y * uj.y;
      tau = 2.0 * uj2 / (nrm2 - aabs * aabs + uj2);
      ujinv = make_double2(uj.x / uj2, -uj.y / uj2);                             // 1 / u_j
    }
    // trailing columns: a <- a - tau u (u^H a) with u = x / u_j (u_j = 1); then new partial norms
    if (tau != 0.0) {
      for (int k = j + 1 + gw; k < Na; k += ngw) {
        double2* a = X + (size_t)k * Ma;
        double sr = 0, si = 0;
        for (int r = j + lane; r < Ma; r += 32) {
          double2 u = make_double2(1.0, 0.0);
          if (r != j) {
            const double2 xv = __ldcg(x + r);
            u = make_double2(xv.x * ujinv.x - xv.y * ujinv.y, xv.x * ujinv.y + xv.y * ujinv.x);
          }
          const double2 av = __ldcg(a + r);
          sr += u.x * av.x + u.y * av.y;      // conj(u) a
          si += u.x * av.y - u.y * av.x;
        }
        sr = wsum(sr);
        si = wsum(si);
        const double tr_ = tau * sr, ti_ = tau * si;
        double nn = 0;
        for (int r = j + lane; r < Ma; r += 32) {
          double2 u = make_double2(1.0, 0.0);
          if (r != j) {
            const double2 xv = __ldcg(x + r);
            u = make_double2(xv.x * ujinv.x - xv.y * ujinv.y, xv.x * ujinv.y + xv.y * ujinv.x);
          }
          double2 av = __ldcg(a + r);
          av.x -= u.x * tr_ - u.y * ti_;
          av.y -= u.x * ti_ + u.y * tr_;
          __stcg(a + r, av);
          if (r > j) nn += av.x * av.x + av.y * av.y;
        }
        nn = wsum(nn);
        if (lane == 0) __stcg(nrm + k, nn);
      }
    }
    cl.sync();                                    // every warp has read column j
    if (gt == 0) {
      __stcg(X + (size_t)j * Ma + j, beta);
      __stcg(nrm + j, 0.0);
    }
    cl.sync();
  }
}

constexpr int QR_SMEM_THREADS = 512;

// The same factorisation with the matrix held in the shared memory of a thread-block cluster.
// Storage column s lives in CTA s % C at local index s / C. Pivoting is logical: the pivot column
// is not moved; it is marked done and its position recorded (qp[j] = p), so R[i, j] is row i of
// storage column qp[j] (i < j) and R[j, j] = beta of that column. Each step needs one cluster
// barrier: every CTA publishes its best remaining column (a double-buffered candidate), reads the
// C candidates and the pivot column (distributed shared memory), and updates its own columns.
// At the end every CTA writes the rows of B = R^H that belong to its columns.
// The partial column norms that pick the pivots are downdated, n <- n - |a_j|^2, and recomputed
// where that cancels below sqrt(eps) of the last exact value (the safeguard of LAPACK's pivoted
// QR); they only choose pivots. The reflector uses the exact norm of the pivot column.
// Dynamic shared memory: X[lq_cap][m_cap] | hv[m_cap] | beta[lq_cap] (double2), nrm[lq_cap] |
// nref[lq_cap] (double), qp[n_cap] | pos[n_cap] | done[lq_cap] (int).
__global__ void __launch_bounds__(QR_SMEM_THREADS, 1)
    k_qrcp_smem(const BondWork* work, int n_work, int lq_cap, int m_cap, int n_cap, int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int w = blockIdx.x / C;
  if (w >= n_work) return;                        // uniform across the cluster
  const BondWork& W = work[w];
  int Ma, Na;
  shape(W, &Ma, &Na);
  if (Na <= 0) return;
  if (Ma > m_cap || Na > n_cap || (Na + C - 1) / C > lq_cap || Ma < Na) {
    if (rank == 0 && threadIdx.x == 0) atomicOr(status, ST_CAPACITY);
    return;
  }
  extern __shared__ double2 sm[];
  double2* X = sm;
  double2* hv = X + (size_t)lq_cap * m_cap;
  double2* betaL = hv + m_cap;
  double* nrm = (double*)(betaL + lq_cap);
  double* nref = nrm + lq_cap;
  int* qp = (int*)(nref + lq_cap);
  int* pos = qp + n_cap;
  int* done = pos + n_cap;
  __shared__ double s_cval[2];
  __shared__ int s_cidx[2];
  __shared__ double s_sc[1];                      // kappa of the step's reflector
  __shared__ double s_red[32];
  __shared__ int s_p;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int Ln = rank < Na ? (Na - rank + C - 1) / C : 0;
  // load the own columns, their norms
  for (int e = tid; e < Ln * Ma; e += blockDim.x) {
    const int l = e / Ma, r = e % Ma;
    X[(size_t)l * m_cap + r] = W.A[r + (size_t)(rank + l * C) * Ma];
  }
  __syncthreads();
  for (int l = wid; l < Ln; l += nw) {
    const double2* a = X + (size_t)l * m_cap;
    double sq = 0;
    for (int r = lane; r < Ma; r += 32) sq += a[r].x * a[r].x + a[r].y * a[r].y;
    sq = wsum(sq);
    if (lane == 0) {
      nrm[l] = sq;
      nref[l] = sq;
      done[l] = 0;
    }
  }
  __syncthreads();
  // local candidate (largest remaining norm, smallest index on ties) into slot par
  auto publish = [&](int par) {
    if (wid == 0) {
      double best = -1.0;
      int bi = 0x7fffffff;
      for (int l = lane; l < Ln; l += 32)
        if (!done[l] && nrm[l] > best) { best = nrm[l]; bi = rank + l * C; }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        s_cval[par] = best;
        s_cidx[par] = bi;
      }
    }
  };
  publish(0);
  cl.sync();
  for (int j = 0; j < Na; ++j) {
    const int par = j & 1;
    // 1. the pivot: best of the C candidates (same values, same order in every CTA)
    if (wid == 0) {
      double best = -1.0;
      int bi = 0x7fffffff;
      if (lane < C) {
        best = *cl.map_shared_rank(&s_cval[par], lane);
        bi = *cl.map_shared_rank(&s_cidx[par], lane);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) s_p = bi;
    }
    __syncthreads();
    const int p = s_p, owner = p % C, lp = p / C;
    const double2* src = cl.map_shared_rank(X, owner) + (size_t)lp * m_cap;
    // 2. the pivot column (rows j..) and its exact squared norm: every CTA sums the same values
    //    in the same order, then derives the Householder scalars with identical arithmetic
    {
      double part = 0;
      for (int r = j + tid; r < Ma; r += blockDim.x) {
        const double2 xv = src[r];
        hv[r] = xv;
        part += xv.x * xv.x + xv.y * xv.y;
      }
      part = wsum(part);
      if (lane == 0) s_red[wid] = part;
    }
    __syncthreads();
    if (tid == 0) {
      // H = I - kappa v v^H with v = x - beta e_j, beta = -phase(alpha) ||x||:
      // v^H v = 2 ||x|| (||x|| + |alpha|), so kappa = 1 / (||x|| (||x|| + |alpha|))
      double nrm2 = 0;
      for (int k = 0; k < nw; ++k) nrm2 += s_red[k];
      const double2 alpha = hv[j];
      const double a2 = alpha.x * alpha.x + alpha.y * alpha.y;
      double kap = 0.0;
      double2 beta = alpha;
      if (nrm2 > 0.0) {
        const double xn = sqrt(nrm2);
        double2 ph = make_double2(1.0, 0.0);
        double aabs = 0.0;
        if (a2 > 0.0) {
          const double ia = rsqrt(a2);
          aabs = a2 * ia;
          ph = make_double2(alpha.x * ia, alpha.y * ia);
        }
        beta = make_double2(-ph.x * xn, -ph.y * xn);
        kap = 1.0 / (xn * (xn + aabs));
        hv[j] = make_double2(ph.x * (aabs + xn), ph.y * (aabs + xn));     // v_j = alpha - beta
      }
      s_sc[0] = kap;
      qp[j] = p;
      if (rank == owner) {
        betaL[lp] = beta;
        done[lp] = 1;
      }
    }
    __syncthreads();
    const double kap = s_sc[0];
    // 3. own remaining columns: a <- a - kappa v (v^H a); partial norms over rows > j
    for (int l = wid; l < Ln; l += nw) {
      if (done[l]) continue;
      double2* a = X + (size_t)l * m_cap;
      if (kap != 0.0) {
        double sr = 0, si = 0;
        for (int r = j + lane; r < Ma; r += 32) {
          const double2 u = hv[r], av = a[r];
          sr = fma(u.x, av.x, fma(u.y, av.y, sr));
          si = fma(u.x, av.y, fma(-u.y, av.x, si));
        }
        const double part = wsum2(sr, si, lane);
        const double tr_ = kap * __shfl_sync(0xffffffffu, part, 0), ti_ = kap * __shfl_sync(0xffffffffu, part, 16);
        for (int r = j + lane; r < Ma; r += 32) {
          const double2 u = hv[r];
          double2 av = a[r];
          av.x -= u.x * tr_ - u.y * ti_;
          av.y -= u.x * ti_ + u.y * tr_;
          a[r] = av;
        }
        __syncwarp();
      }
      const double2 ajv = a[j];
      double nn = nrm[l] - (ajv.x * ajv.x + ajv.y * ajv.y);
      if (nn <= 1.4901161193847656e-8 * nref[l]) {     // cancellation: recompute
        double sq = 0;
        for (int r = j + 1 + lane; r < Ma; r += 32) sq += a[r].x * a[r].x + a[r].y * a[r].y;
        nn = wsum(sq);
        if (lane == 0) nref[l] = nn;
      }
      if (lane == 0) nrm[l] = nn;
    }
    __syncthreads();
    publish(par ^ 1);
    cl.sync();                                    // candidates published; pivot column reads done
  }
  // permutation (every CTA holds the same qp), B = R^H rows of the own columns
  for (int j = tid; j < Na; j += blockDim.x) pos[qp[j]] = j;
  if (rank == 0)
    for (int j = tid; j < Na; j += blockDim.x) W.qperm[j] = qp[j];
  __syncthreads();
  for (int l = wid; l < Ln; l += nw) {
    const int s = rank + l * C, i = pos[s];
    const double2* a = X + (size_t)l * m_cap;
    for (int c = lane; c < Na; c += 32) {
      double2 v = make_double2(0.0, 0.0);           // B[i, c] = conj(R[c, i])
      if (c < i) v = make_double2(a[c].x, -a[c].y);
      else if (c == i) v = make_double2(betaL[l].x, -betaL[l].y);
      W.G64[i + (size_t)c * Na] = v;
    }
  }
  cl.sync();                                      // no CTA leaves while its memory may be read
}

constexpr int QRG_THREADS = 512;
constexpr int QRG_WARPS = QRG_THREADS / 32;
constexpr int QRG_MAX_ITEMS = 256;
constexpr int QRG_RC = 8;                 // rows per lane held in registers: Ma <= 256

// The same factorisation for every matrix of a layer on the whole GPU (a cooperative launch, one
// 512-thread CTA per SM): the concatenated columns of all matrices are split into equal ranges,
// one range per CTA and one column per warp. A warp keeps its column's rows j.. in registers (a
// one-row shift between steps) and writes them back to the workspace (Y64), where other CTAs
// read pivot columns. Step j: every CTA picks the pivot of each matrix it holds columns of from
// the partial norms (same values, same order everywhere), reads the pivot column and its exact
// norm, and its warps apply the reflector; one grid barrier per step. The partial norms are
// double-buffered (aux and sig alternate: step j reads one and writes the other, so a CTA still
// choosing step j's pivot never sees step j+1's values); finished columns write -1. The pivot's owner records qperm[j] and beta_j (in V, free until the finish).
// Finally every warp writes its column of B = R^H.
__global__ void __launch_bounds__(QRG_THREADS, 1)
    k_qrcp_grid(const BondWork* work, int n_work, GridSync gs, int* status) {
  extern __shared__ double2 hv[];
  __shared__ int s_off[QRG_MAX_ITEMS + 1];
  __shared__ int s_Ma[QRG_MAX_ITEMS];
  __shared__ int s_maxna;
  __shared__ double s_red[QRG_WARPS];
  __shared__ double s_kap;
  __shared__ int s_p, s_own;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (n_work > QRG_MAX_ITEMS) {
    if (blockIdx.x == 0 && tid == 0) atomicOr(status, ST_CAPACITY);
    return;
  }
  if (tid == 0) {
    int o = 0, mx = 0;
    for (int w = 0; w < n_work; ++w) {
      int Ma, Na;
      shape(work[w], &Ma, &Na);
      if (Ma > 32 * QRG_RC) {                // the host never launches such a layer here
        if (blockIdx.x == 0) atomicOr(status, ST_CAPACITY);
        Na = 0;
      }
      s_off[w] = o;
      s_Ma[w] = Ma;
      o += Na;
      mx = max(mx, Na);
    }
    s_off[n_work] = o;
    s_maxna = mx;
  }
  __syncthreads();
  const int total = s_off[n_work];
  const int per = (total + gridDim.x - 1) / gridDim.x;
  if (per > QRG_WARPS) {
    if (blockIdx.x == 0 && tid == 0) atomicOr(status, ST_CAPACITY);
    return;                                   // uniform: every CTA sees the same total
  }
  const int g0 = min(total, (int)blockIdx.x * per), g1 = min(total, g0 + per);
  // this warp's column (w_me, s_me), if any
  const int gme = g0 + wid;
  const bool have = wid < per && gme < g1;
  int w_me = 0;
  if (have) {
    int lo = 0, hi = n_work - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_off[mid] <= gme) lo = mid;
      else hi = mid - 1;
    }
    w_me = lo;
  }
  const int s_me = gme - s_off[w_me];
  const int Ma_me = have ? s_Ma[w_me] : 0;
  double2 c[QRG_RC];
  double nrm_me = 0, nref_me = 0;
  bool done = !have;
  if (have) {
    const BondWork& W = work[w_me];
    double sq = 0;
#pragma unroll
    for (int k = 0; k < QRG_RC; ++k) {
      const int r = lane + 32 * k;
      c[k] = make_double2(0.0, 0.0);
      if (r < Ma_me) {
        c[k] = W.A[r + (size_t)s_me * Ma_me];
        __stcg(W.Y64 + r + (size_t)s_me * Ma_me, c[k]);
        sq += c[k].x * c[k].x + c[k].y * c[k].y;
      }
    }
    sq = wsum(sq);
    nrm_me = nref_me = sq;
    if (lane == 0) __stcg(W.aux + s_me, sq);       // step 0 reads aux
  }
  // the matrices this CTA holds columns of: w_lo..w_hi (none when g0 == g1)
  auto item_of = [&](int g) {
    int lo = 0, hi = n_work - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_off[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  };
  const int w_lo = g0 < g1 ? item_of(g0) : 0;
  const int w_hi = g0 < g1 ? item_of(g1 - 1) : -1;
  if (!grid_barrier(gs, status)) return;
  const int maxna = s_maxna;
  for (int j = 0; j < maxna; ++j) {
    for (int w = w_lo; w <= w_hi; ++w) {
      const int Na = s_off[w + 1] - s_off[w], Ma = s_Ma[w];
      if (j >= Na) continue;                  // uniform across the CTA
      const BondWork& W = work[w];
      const double2* X = W.Y64;
      const double* nrm_cur = (j & 1) ? W.sig : W.aux;
      double* nrm_nxt = (j & 1) ? W.aux : W.sig;
      // (a) pivot: largest remaining partial norm, smallest index on ties (Na <= 256: all loads
      //     of a lane are issued before the first comparison)
      if (wid == 0) {
        double best = -1.0;
        int bi = 0x7fffffff;
        double v[QRG_RC];
#pragma unroll
        for (int k = 0; k < QRG_RC; ++k) {
          const int i = lane + 32 * k;
          v[k] = i < Na ? __ldcg(nrm_cur + i) : -2.0;
        }
#pragma unroll
        for (int k = 0; k < QRG_RC; ++k)
          if (v[k] > best) { best = v[k]; bi = lane + 32 * k; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) s_p = bi;
      }
      __syncthreads();
      const int p = s_p;
      // (b) the pivot column (rows j..) and its exact norm, summed in the same order everywhere
      {
        double part = 0;
        for (int r = j + tid; r < Ma; r += blockDim.x) {
          const double2 xv = __ldcg(X + r + (size_t)p * Ma);
          hv[r] = xv;
          part += xv.x * xv.x + xv.y * xv.y;
        }
        part = wsum(part);
        if (lane == 0) s_red[wid] = part;
      }
      __syncthreads();
      if (tid == 0) {
        double nrm2 = 0;
        for (int k = 0; k < QRG_WARPS; ++k) nrm2 += s_red[k];
        const double2 alpha = hv[j];
        const double a2 = alpha.x * alpha.x + alpha.y * alpha.y;
        double kap = 0.0;
        double2 beta = alpha;
        if (nrm2 > 0.0) {
          const double xn = sqrt(nrm2);
          double2 ph = make_double2(1.0, 0.0);
          double aabs = 0.0;
          if (a2 > 0.0) {
            const double ia = rsqrt(a2);
            aabs = a2 * ia;
            ph = make_double2(alpha.x * ia, alpha.y * ia);
          }
          beta = make_double2(-ph.x * xn, -ph.y * xn);
          kap = 1.0 / (xn * (xn + aabs));
          hv[j] = make_double2(ph.x * (aabs + xn), ph.y * (aabs + xn));
        }
        s_kap = kap;
        const int gp = s_off[w] + p;
        s_own = -1;
        if (gp >= g0 && gp < g1) {              // this CTA owns the pivot column
          s_own = gp - g0;
          __stcg(W.qperm + j, p);
          __stcg(W.V + j, beta);
        }
      }
      __syncthreads();
      const double kap = s_kap;
      if (have && w_me == w) {
        if (wid == s_own) done = true;
        if (done) {
          if (lane == 0) __stcg(nrm_nxt + s_me, -1.0);
        } else {
          double2* a = W.Y64 + (size_t)s_me * Ma;
          if (kap != 0.0) {
            double sr = 0, si = 0;
#pragma unroll
            for (int k = 0; k < QRG_RC; ++k) {
              const int r = j + lane + 32 * k;
              if (r < Ma) {
                const double2 u = hv[r];
                sr = fma(u.x, c[k].x, fma(u.y, c[k].y, sr));
                si = fma(u.x, c[k].y, fma(-u.y, c[k].x, si));
              }
            }
            const double part = wsum2(sr, si, lane);
            const double tr_ = kap * __shfl_sync(0xffffffffu, part, 0);
            const double ti_ = kap * __shfl_sync(0xffffffffu, part, 16);
#pragma unroll
            for (int k = 0; k < QRG_RC; ++k) {
              const int r = j + lane + 32 * k;
              if (r < Ma) {
                const double2 u = hv[r];
                c[k].x -= u.x * tr_ - u.y * ti_;
                c[k].y -= u.x * ti_ + u.y * tr_;
                __stcg(a + r, c[k]);
              }
            }
          }
          // partial norm over rows > j: downdated, recomputed where that cancels
          const double2 ajv = make_double2(__shfl_sync(0xffffffffu, c[0].x, 0), __shfl_sync(0xffffffffu, c[0].y, 0));
          double nn = nrm_me - (ajv.x * ajv.x + ajv.y * ajv.y);
          if (nn <= 1.4901161193847656e-8 * nref_me) {
            double sq = 0;
#pragma unroll
            for (int k = 0; k < QRG_RC; ++k) {
              const int r = j + lane + 32 * k;
              if (r > j && r < Ma) sq += c[k].x * c[k].x + c[k].y * c[k].y;
            }
            nn = wsum(sq);
            nref_me = nn;
          }
          nrm_me = nn;
          if (lane == 0) __stcg(nrm_nxt + s_me, nn);
          // registers move one row: lane l takes row j+1+l+32k
#pragma unroll
          for (int k = 0; k < QRG_RC; ++k) {
            const double2 nxt = k + 1 < QRG_RC ? c[k + 1] : make_double2(0.0, 0.0);
            const double2 own = c[k];
            // lane l receives from lane l+1 its row j+1+l+32k; lane 31 receives lane 0's next row
            const double xs = __shfl_sync(0xffffffffu, lane == 0 ? nxt.x : own.x, (lane + 1) & 31);
            const double ys = __shfl_sync(0xffffffffu, lane == 0 ? nxt.y : own.y, (lane + 1) & 31);
            c[k] = make_double2(xs, ys);
          }
        }
      }
      __syncthreads();                          // hv is rewritten by the next matrix
    }
    if (!grid_barrier(gs, status)) return;
  }
  // B = R^H: column c of B is row c of R, B[i, c] = conj(R[c, i]), R[c, qperm[i]] = X[c, qperm[i]]
  if (have) {
    const BondWork& W = work[w_me];
    const int Na = s_off[w_me + 1] - s_off[w_me], Ma = Ma_me, cc = s_me;
    for (int i = lane; i < Na; i += 32) {
      double2 v = make_double2(0.0, 0.0);
      if (cc < i) {
        const double2 r = __ldcg(W.Y64 + cc + (size_t)__ldcg(W.qperm + i) * Ma);
        v = make_double2(r.x, -r.y);
      } else if (cc == i) {
        const double2 b = __ldcg(W.V + cc);
        v = make_double2(b.x, -b.y);
      }
      W.G64[i + (size_t)cc * Na] = v;
    }
  }
}

// B = R^H (Na x Na, col-major, lower triangular) from the upper triangle of the QR workspace
__global__ void k_qrcp_rh(const BondWork* work, int n_work) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  shape(W, &Ma, &Na);
  const size_t tot = (size_t)Na * Na;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % Na), c = (int)(idx / Na);     // B[i, c] = conj(R[c, i]) for c <= i
    double2 v = make_double2(0.0, 0.0);
    if (c <= i) {
      const double2 r = W.Y64[c + (size_t)i * Ma];
      v = make_double2(r.x, -r.y);
    }
    W.G64[idx] = v;
  }
}

// V_D = P U': V[qperm[k], c] = U'[k, c] (U' = the normalised columns of B after the Jacobi)
__global__ void k_qrcp_vd(const BondWork* work, int n_work) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  shape(W, &Ma, &Na);
  const size_t tot = (size_t)Na * Na;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % Na), c = (int)(idx / Na);
    W.V[W.qperm[k] + (size_t)c * Na] = W.G64[idx];
  }
}

// U_D = (D V_D) / sigma, column by column (Y64 holds D V_D)
__global__ void k_qrcp_ud(const BondWork* work, int n_work) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  shape(W, &Ma, &Na);
  const size_t tot = (size_t)Ma * Na;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / Ma);
    const double s = W.sig[c];
    const double2 y = W.Y64[idx];
    W.A[idx] = s > 0.0 ? make_double2(y.x / s, y.y / s) : make_double2(0.0, 0.0);
  }
}

static cudaLaunchConfig_t qr_cfg(int n_work, int cluster, cudaStream_t st, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_work * cluster, 1, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

static size_t qr_smem_bytes(int lq, int m_cap, int n_cap) {
  return sizeof(double2) * ((size_t)lq * m_cap + m_cap + lq) + sizeof(double) * 2 * lq +
         sizeof(int) * (2 * (size_t)n_cap + lq);
}

// Cluster size for the shared-memory factorisation of matrices up to m_cap x n_cap; 0 if they do
// not fit (the global-memory kernel is used then).
int qrcp_smem_cluster(int m_cap, int n_cap) {
  cudaFuncSetAttribute(k_qrcp_smem, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int c = 16; c >= 2; c >>= 1) {
    const int lq = (n_cap + c - 1) / c;
    const size_t bytes = qr_smem_bytes(lq, m_cap, n_cap);
    if (bytes > 200 * 1024) return 0;
    if (cudaFuncSetAttribute(k_qrcp_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c, 1, 1);
    cfg.blockDim = dim3(QR_SMEM_THREADS, 1, 1);
    cfg.dynamicSmemBytes = bytes;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_qrcp_smem, &cfg) == cudaSuccess && n > 0) return c;
    cudaGetLastError();
  }
  return 0;
}

int qrcp_grid_ok() {
  int a = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_qrcp_grid, QRG_THREADS, 32 * QRG_RC * sizeof(double2)) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return a >= 1;
}

int qrcp_grid_fits(int n_work, int m_cap, int total_cols_cap, int blocks) {
  return n_work <= QRG_MAX_ITEMS && m_cap <= 32 * QRG_RC && blocks > 0 &&
         (total_cols_cap + blocks - 1) / blocks <= QRG_WARPS;
}

void launch_qrcp_grid(const BondWork* work, int n_work, int blocks, unsigned* sync3, int* status, cudaStream_t st) {
  cudaMemsetAsync(sync3, 0, sizeof(unsigned), st);
  cudaMemsetAsync(sync3 + 2, 0, sizeof(unsigned), st);
  GridSync gs{sync3, (int*)(sync3 + 2), GRID_WAIT_LIMIT_CYCLES};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks, 1, 1);
  cfg.blockDim = dim3(QRG_THREADS, 1, 1);
  cfg.dynamicSmemBytes = 32 * QRG_RC * sizeof(double2);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_qrcp_grid, work, n_work, gs, status);
}

int qrcp_cluster_size(int want) {
  cudaFuncSetAttribute(k_qrcp, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int c = 16; c >= 1; c >>= 1) {
    if (c > want) continue;
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = qr_cfg(1, c, 0, at);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_qrcp, &cfg) == cudaSuccess && n > 0) return c;
    cudaGetLastError();
  }
  return 1;
}

void launch_qrcp_precondition(const BondWork* work, int n_work, int cluster, int smem_cluster, int k_cap, int m_cap,
                              int* status, cudaStream_t st) {
  cudaLaunchAttribute at[1];
  if (smem_cluster > 0) {
    const int lq = (k_cap + smem_cluster - 1) / smem_cluster;
    cudaLaunchConfig_t cfg = qr_cfg(n_work, smem_cluster, st, at);
    cfg.blockDim = dim3(QR_SMEM_THREADS, 1, 1);
    cfg.dynamicSmemBytes = qr_smem_bytes(lq, m_cap, k_cap);
    cudaLaunchKernelEx(&cfg, k_qrcp_smem, work, n_work, lq, m_cap, k_cap, status);
    return;
  }
  cudaLaunchConfig_t cfg = qr_cfg(n_work, cluster, st, at);
  cudaLaunchKernelEx(&cfg, k_qrcp, work, n_work);
  k_qrcp_rh<<<dim3(128, n_work), 256, 0, st>>>(work, n_work);
}

void launch_qrcp_finish(const BondWork* work, int n_work, int k_cap, int m_cap, cudaStream_t st) {
  k_qrcp_vd<<<dim3(128, n_work), 256, 0, st>>>(work, n_work);
  launch_mix_gemm_av(work, n_work, k_cap, m_cap, st);
  k_qrcp_ud<<<dim3(128, n_work), 256, 0, st>>>(work, n_work);
}

}  // namespace ptk
