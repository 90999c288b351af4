// QR-preconditioned one-sided Jacobi for the bond SVD (App. A.2).
//
// A one-sided Jacobi on a rank-deficient, strongly graded D needs many sweeps (17-23 on the
// five-site chain's 256x256 blocks); after a column-pivoted QR, D P = Q R, the same Jacobi on R^H
// converges in ~8 (Drmac and Veselic's preconditioning). Here:
//   1. the pivoted Householder QR of D, with B = R^H written directly: on the whole GPU
//      (k_qrcp_grid) where a layer's columns fit one per warp, else one thread-block cluster per
//      matrix with the columns in shared memory or, for large matrices, in global memory
//      (k_qrcp_cl);
//   2. the grid Jacobi on B gives B = U' S V'^H, i.e. R = V' S U'^H and D = (Q V') S (P U')^H;
//   3. after the truncation, k_qrcp_vd: V_D = P U' (rows permuted back) on the kept columns;
//   4. U_D = D V_D S^{-1} on the kept columns by an FP64 GEMM (k_mix_gemm) and a column scaling
//      (k_qrcp_ud). Its error in column c is ~eps ||D|| / s_c, and that column enters the truncated
//      state scaled by s_c, so the state error stays at rounding level; Q is never formed.
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

constexpr int QR_SMEM_THREADS = 512;

// The same factorisation with one thread-block cluster per matrix. Storage column s belongs to CTA
// s % C at local index s / C; GL = false keeps the columns in the CTAs' shared memory (pivot columns
// read through distributed shared memory), GL = true leaves them in the workspace Y64 (global,
// through L2) for matrices too large for shared memory. Pivoting is logical: the pivot column is
// not moved; it is marked done and its position recorded (qp[j] = p), so R[i, j] is row i of
// storage column qp[j] (i < j) and R[j, j] = beta of that column. Each step needs one cluster
// barrier: every CTA publishes its best remaining column (a double-buffered candidate), reads the
// C candidates and the pivot column, and updates its own columns. At the end every CTA writes the
// rows of B = R^H that belong to its columns.
// The partial column norms that pick the pivots are downdated, n <- n - |a_j|^2, and recomputed
// where that cancels below sqrt(eps) of the last exact value (the safeguard of LAPACK's pivoted
// QR); they only choose pivots. The reflector uses the exact norm of the pivot column.
// Rank-revealing stop: the factorisation ends at the first step j whose pivot column (the largest
// remaining one) has an exact norm^2 <= tau^2 ||D||_F^2, with tau the noise level of D: u = 2^-53
// when D was formed in FP64 (the level below which the Jacobi does not rotate a column either),
// 2^-40 for the fixed-point-slice tensor-core product (whose error in D's null space is ~3e-14 of
// ||D||_F). Every remaining column is then noise, and the trailing block R22 they form,
// ||R22||_F <= sqrt(n) tau ||D||_F, is dropped -- for tau = u a perturbation within the backward
// error of any FP64 SVD, for 2^-40 one far below every truncation threshold (>= 1e-10 sigma_1). R is then k x n (k = j, recorded in info[8]) and
// B = R^H is n x k, so the Jacobi runs on k columns. (The workloads' D are often exactly rank
// deficient: a conserved magnetisation leaves ~n/4 nonzero singular values.)
// Dynamic shared memory: [X[lq_cap][m_cap] if !GL] | hv[m_cap] | beta[lq_cap] (double2),
// nrm[lq_cap] | nref[lq_cap] (double), qp[n_cap] | pos[n_cap] | done[lq_cap] (int).
template <bool GL>
__global__ void __launch_bounds__(QR_SMEM_THREADS, 1)
    k_qrcp_cl(const BondWork* work, int n_work, int lq_cap, int m_cap, int n_cap, double tau2, int kmax,
              int* status) {
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
  double2* X = sm;                                // local columns (shared memory mode only)
  double2* hv = GL ? sm : X + (size_t)lq_cap * m_cap;
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
  __shared__ double s_fro;                        // this CTA's share of ||D||_F^2
  __shared__ double s_thr2;                       // the noise floor u^2 ||D||_F^2 (tid 0)
  __shared__ int s_stop, s_k;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int Ln = rank < Na ? (Na - rank + C - 1) / C : 0;
  // local column l, its element loads and stores (L2-coherent in global mode)
  auto colp = [&](int l) -> double2* {
    return GL ? W.Y64 + (size_t)(rank + l * C) * Ma : X + (size_t)l * m_cap;
  };
  auto ld = [&](const double2* q) -> double2 { return GL ? __ldcg(q) : *q; };
  auto st = [&](double2* q, double2 v) {
    if (GL) __stcg(q, v);
    else *q = v;
  };
  // load the own columns, their norms
  for (int e = tid; e < Ln * Ma; e += blockDim.x) {
    const int l = e / Ma, r = e % Ma;
    st(colp(l) + r, W.A[r + (size_t)(rank + l * C) * Ma]);
  }
  __syncthreads();
  for (int l = wid; l < Ln; l += nw) {
    const double2* a = colp(l);
    double sq = 0;
    for (int r = lane; r < Ma; r += 32) {
      const double2 v = ld(a + r);
      sq += v.x * v.x + v.y * v.y;
    }
    sq = wsum(sq);
    if (lane == 0) {
      nrm[l] = sq;
      nref[l] = sq;
      done[l] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double f = 0;
    for (int l = 0; l < Ln; ++l) f += nrm[l];
    s_fro = f;
    s_stop = 0;
    s_k = Na;
  }
  // local candidate (largest remaining norm, smallest index on ties) into slot par
  auto publish = [&](int par) {
    if (wid == 0) {
      double best = -1.0;
      int bi = 0x7fffffff;
      // a NaN norm counts as 0, so an unfinished column is always chosen (the index stays valid)
      for (int l = lane; l < Ln; l += 32) {
        const double nl = nrm[l] == nrm[l] ? nrm[l] : 0.0;
        if (!done[l] && nl > best) { best = nl; bi = rank + l * C; }
      }
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
  if (threadIdx.x == 0) {
    // ||D||_F^2 from the C shares, summed in the same order in every CTA
    double f = 0;
    for (int r = 0; r < C; ++r) f += *cl.map_shared_rank(&s_fro, r);
    s_thr2 = tau2 * f;                             // tau^2 ||D||_F^2
  }
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
    const double2* src;
    if constexpr (GL) src = W.Y64 + (size_t)p * Ma;
    else src = cl.map_shared_rank(X, owner) + (size_t)lp * m_cap;
    // 2. the pivot column (rows j..) and its exact squared norm: every CTA sums the same values
    //    in the same order, then derives the Householder scalars with identical arithmetic
    {
      double part = 0;
      for (int r = j + tid; r < Ma; r += blockDim.x) {
        const double2 xv = ld(src + r);
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
      if (nrm2 <= s_thr2 || j >= kmax) {
        // every remaining column is at the noise floor (or the caller's step limit): stop, the same
        // decision in every CTA
        s_stop = 1;
        s_k = j;
      } else {
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
    }
    __syncthreads();
    if (s_stop) break;                            // uniform across the cluster
    const double kap = s_sc[0];
    // 3. own remaining columns: a <- a - kappa v (v^H a); partial norms over rows > j
    for (int l = wid; l < Ln; l += nw) {
      if (done[l]) continue;
      double2* a = colp(l);
      if (kap != 0.0) {
        double sr = 0, si = 0;
        for (int r = j + lane; r < Ma; r += 32) {
          const double2 u = hv[r], av = ld(a + r);
          sr = fma(u.x, av.x, fma(u.y, av.y, sr));
          si = fma(u.x, av.y, fma(-u.y, av.x, si));
        }
        const double part = wsum2(sr, si, lane);
        const double tr_ = kap * __shfl_sync(0xffffffffu, part, 0), ti_ = kap * __shfl_sync(0xffffffffu, part, 16);
        for (int r = j + lane; r < Ma; r += 32) {
          const double2 u = hv[r];
          double2 av = ld(a + r);
          av.x -= u.x * tr_ - u.y * ti_;
          av.y -= u.x * ti_ + u.y * tr_;
          st(a + r, av);
        }
        __syncwarp();
      }
      const double2 ajv = ld(a + j);
      double nn = nrm[l] - (ajv.x * ajv.x + ajv.y * ajv.y);
      if (nn <= 1.4901161193847656e-8 * nref[l]) {     // cancellation: recompute
        double sq = 0;
        for (int r = j + 1 + lane; r < Ma; r += 32) {
          const double2 v = ld(a + r);
          sq += v.x * v.x + v.y * v.y;
        }
        nn = wsum(sq);
        if (lane == 0) nref[l] = nn;
      }
      if (lane == 0) nrm[l] = nn;
    }
    __syncthreads();
    publish(par ^ 1);
    cl.sync();                                    // candidates published; pivot column reads done
  }
  // permutation (every CTA holds the same qp): the k pivots in order, then the remaining columns
  // by index; B = R^H (Na x k) rows of the own columns
  const int kq = s_k;
  for (int j = tid; j < Na; j += blockDim.x) pos[j] = -1;
  __syncthreads();
  for (int j = tid; j < kq; j += blockDim.x) pos[qp[j]] = j;
  __syncthreads();
  if (wid == 0) {
    int i = kq;
    for (int s0 = 0; s0 < Na; s0 += 32) {
      const int s = s0 + lane;
      const bool rem = s < Na && pos[s] < 0;
      const unsigned bal = __ballot_sync(0xffffffffu, rem);
      if (rem) {
        const int at = i + __popc(bal & ((1u << lane) - 1u));
        pos[s] = at;
        qp[at] = s;
      }
      i += __popc(bal);
    }
  }
  __syncthreads();
  if (rank == 0) {
    for (int j = tid; j < Na; j += blockDim.x) W.qperm[j] = qp[j];
    if (tid == 0) W.info[8] = kq;
  }
  for (int l = wid; l < Ln; l += nw) {
    const int s = rank + l * C, i = pos[s];
    const double2* a = colp(l);
    for (int c = lane; c < kq; c += 32) {
      double2 v = make_double2(0.0, 0.0);           // B[i, c] = conj(R[c, i])
      if (c < i) {
        const double2 x = ld(a + c);
        v = make_double2(x.x, -x.y);
      }
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
// The same rank-revealing stop as k_qrcp_cl ends a matrix at the first pivot at the noise floor.
// Finally every warp writes the row of B = R^H (Na x k) that belongs to its column.
__global__ void __launch_bounds__(QRG_THREADS, 1)
    k_qrcp_grid(const BondWork* work, int n_work, GridSync gs, double tau2, int kmax, int* status) {
  extern __shared__ double2 hv[];
  __shared__ int s_off[QRG_MAX_ITEMS + 1];
  __shared__ int s_Ma[QRG_MAX_ITEMS];
  __shared__ int s_maxna;
  __shared__ double s_red[QRG_WARPS];
  __shared__ double s_kap;
  __shared__ int s_p, s_own, s_stopnow;
  __shared__ double s_thr2[QRG_MAX_ITEMS];  // u^2 ||D||_F^2 of the matrices this CTA holds
  __shared__ int s_kst[QRG_MAX_ITEMS];      // their stop step (Na if never)
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
  // ||D||_F^2 of every matrix this CTA holds columns of, summed in the same order everywhere
  for (int w = w_lo + wid; w <= w_hi; w += QRG_WARPS) {
    const int Na = s_off[w + 1] - s_off[w];
    double f = 0;
    for (int i = lane; i < Na; i += 32) f += __ldcg(work[w].aux + i);
    f = wsum(f);
    if (lane == 0) {
      s_thr2[w] = tau2 * f;                     // tau^2 ||D||_F^2
      s_kst[w] = Na;
    }
  }
  __syncthreads();
  int my_pos = -1;                            // the step at which this warp's column was pivoted
  const int maxna = s_maxna;
  for (int j = 0; j < maxna; ++j) {
    for (int w = w_lo; w <= w_hi; ++w) {
      const int Na = s_off[w + 1] - s_off[w], Ma = s_Ma[w];
      if (j >= s_kst[w]) continue;            // uniform across the CTA and across CTAs
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
          if (!(v[k] == v[k])) v[k] = 0.0;        // NaN: still a valid unfinished column
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
        s_stopnow = 0;
        if (nrm2 <= s_thr2[w] || j >= kmax) {
          // every remaining column is at the noise floor (or the caller's step limit): this matrix
          // stops at rank j
          s_stopnow = 1;
          s_kst[w] = j;
        } else {
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
      }
      __syncthreads();
      if (s_stopnow) continue;                  // uniform; nothing reads hv any more this step
      const double kap = s_kap;
      if (have && w_me == w) {
        if (wid == s_own && !done) {
          done = true;
          my_pos = j;
        }
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
  // B = R^H (Na x k): this warp's column s sits at position i of the pivot order (its step, or for
  // a column never pivoted k + its rank among those by index); row i of B is
  // B[i, c] = conj(R[c, i]) = conj(X[c, s]) for c < i, conj(beta_i) at c = i (i < k), 0 beyond.
  if (have) {
    const BondWork& W = work[w_me];
    const int Na = s_off[w_me + 1] - s_off[w_me], Ma = Ma_me, sc = s_me, kq = s_kst[w_me];
    int i = my_pos;
    if (i < 0) {
      // the step-k norm buffer holds -1 for every pivoted column and >= 0 for the rest
      const double* nb = (kq & 1) ? W.sig : W.aux;
      int before = 0;
      for (int t0 = 0; t0 < sc; t0 += 32) {
        const int t = t0 + lane;
        const bool rem = t < sc && __ldcg(nb + t) >= 0.0;
        before += __popc(__ballot_sync(0xffffffffu, rem));
      }
      i = kq + before;
      if (lane == 0) __stcg(W.qperm + i, sc);
    }
    if (sc == 0 && lane == 0) W.info[8] = kq;
    for (int c = lane; c < kq; c += 32) {
      double2 v = make_double2(0.0, 0.0);
      if (c < i) {
        const double2 r = __ldcg(W.Y64 + c + (size_t)sc * Ma);
        v = make_double2(r.x, -r.y);
      } else if (c == i) {
        const double2 b = __ldcg(W.V + c);
        v = make_double2(b.x, -b.y);
      }
      W.G64[i + (size_t)c * Na] = v;
    }
  }
}

// The finish forms only the columns the truncation keeps (it runs after k_truncate): kept column c
// is Jacobi column perm[c], c < chi = the bond's new dimension.
// V_D = P U' on the kept columns: V[qperm[r], perm[c]] = U'[r, perm[c]] (U' = the normalised columns
// of B after the Jacobi)
__global__ void k_qrcp_vd(const BondWork* work, int n_work, const int* lam_chi) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  shape(W, &Ma, &Na);
  const int kept = min(lam_chi[W.lam_l + 1], Na);
  const size_t tot = (size_t)Na * kept;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % Na), col = W.perm[idx / Na];
    W.V[W.qperm[r] + (size_t)col * Na] = W.G64[r + (size_t)col * Na];
  }
}

// U_D = (D V_D) / sigma on the kept columns (Y64 holds D V_D in kept order)
__global__ void k_qrcp_ud(const BondWork* work, int n_work, const int* lam_chi) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  shape(W, &Ma, &Na);
  const int kept = min(lam_chi[W.lam_l + 1], Na);
  const size_t tot = (size_t)Ma * kept;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
    const int col = W.perm[idx / Ma];
    const double s = W.sig[col];
    const double2 y = W.Y64[idx];
    W.A[idx % Ma + (size_t)col * Ma] = s > 0.0 ? make_double2(y.x / s, y.y / s) : make_double2(0.0, 0.0);
  }
}

static cudaLaunchConfig_t qr_cfg(int n_work, int cluster, cudaStream_t st, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_work * cluster, 1, 1);
  cfg.blockDim = dim3(QR_SMEM_THREADS, 1, 1);
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

static size_t qr_smem_bytes(int lq, int m_cap, int n_cap, bool gl) {
  return sizeof(double2) * ((gl ? 0 : (size_t)lq * m_cap) + m_cap + lq) + sizeof(double) * 2 * lq +
         sizeof(int) * (2 * (size_t)n_cap + lq);
}

// Largest cluster (16, 8, ... down to `lowest`) for which the factorisation of matrices up to
// m_cap x n_cap fits (shared memory per CTA, co-scheduling); 0 if none does.
template <bool GL>
static int qr_pick_cluster(int m_cap, int n_cap, int want, int lowest) {
  cudaFuncSetAttribute(k_qrcp_cl<GL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int c = 16; c >= lowest; c >>= 1) {
    if (c > want) continue;
    const int lq = (n_cap + c - 1) / c;
    const size_t bytes = qr_smem_bytes(lq, m_cap, n_cap, GL);
    if (bytes > 200 * 1024) {
      if (GL) return 0;
      continue;
    }
    if (cudaFuncSetAttribute(k_qrcp_cl<GL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = qr_cfg(1, c, 0, at);
    cfg.dynamicSmemBytes = bytes;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_qrcp_cl<GL>, &cfg) == cudaSuccess && n > 0) return c;
    cudaGetLastError();
  }
  return 0;
}

// Cluster size for the shared-memory factorisation of matrices up to m_cap x n_cap; 0 if they do
// not fit (the columns then stay in global memory).
int qrcp_smem_cluster(int m_cap, int n_cap) { return qr_pick_cluster<false>(m_cap, n_cap, 16, 2); }

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

void launch_qrcp_grid(const BondWork* work, int n_work, int blocks, unsigned* sync3, double tau2, int kmax,
                      int* status, cudaStream_t st) {
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
  cudaLaunchKernelEx(&cfg, k_qrcp_grid, work, n_work, gs, tau2, kmax, status);
}

// Cluster size for the global-memory variant (at most `want` CTAs per matrix; 1 at the least).
int qrcp_cluster_size(int want, int m_cap, int n_cap) {
  const int c = qr_pick_cluster<true>(m_cap, n_cap, want, 1);
  return c > 0 ? c : 1;
}

void launch_qrcp_precondition(const BondWork* work, int n_work, int cluster, int smem_cluster, int k_cap, int m_cap,
                              double tau2, int kmax, int* status, cudaStream_t st) {
  cudaLaunchAttribute at[1];
  const bool gl = smem_cluster <= 0;
  const int c = gl ? cluster : smem_cluster;
  const int lq = (k_cap + c - 1) / c;
  cudaLaunchConfig_t cfg = qr_cfg(n_work, c, st, at);
  cfg.dynamicSmemBytes = qr_smem_bytes(lq, m_cap, k_cap, gl);
  if (gl) cudaLaunchKernelEx(&cfg, k_qrcp_cl<true>, work, n_work, lq, m_cap, k_cap, tau2, kmax, status);
  else cudaLaunchKernelEx(&cfg, k_qrcp_cl<false>, work, n_work, lq, m_cap, k_cap, tau2, kmax, status);
}

void launch_qrcp_finish(const BondWork* work, int n_work, int k_cap, int m_cap, const int* lam_chi,
                        cudaStream_t st) {
  k_qrcp_vd<<<dim3(128, n_work), 256, 0, st>>>(work, n_work, lam_chi);
  launch_mix_gemm_av(work, n_work, k_cap, m_cap, lam_chi, st);
  k_qrcp_ud<<<dim3(128, n_work), 256, 0, st>>>(work, n_work, lam_chi);
}

}  // namespace ptk
