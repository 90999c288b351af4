// Whole-GPU one-sided Jacobi SVD for all bond matrices of one layer (App. A.2).
//
// The SVD is bound by FP64 arithmetic (1.2 TFLOP/s on GB300, ~7.9 GFLOP/s per SM), so every SM
// must work on it even when a layer has only two bonds. One cooperative launch (one 512-thread
// CTA per SM) processes every matrix of the layer. The columns are grouped in blocks of two and a
// round-robin tournament runs over the blocks: in each round the block pairs of all matrices form
// one task list, each task handled by a slot of 8 warps (two groups of 4, one warp per SM
// sub-partition in each, the rows split across them) that runs the task's four cross pairs (and,
// in the first round of a sweep, the pair inside each block) in sub-rounds; a grid barrier
// separates the rounds. Partial sums are combined in a fixed order, so results are bitwise
// reproducible. Every barrier wait has a time limit: on expiry the kernel records ST_TIMEOUT,
// raises an abort flag that releases every other CTA, and returns.
//
// on_b = 1: the matrix is R^H left by the pivoted QR (qrcp.cu); only its left vectors are wanted
// there, so the right factor is not accumulated. on_b = 2: the l x l triangular factor of the fast
// path's randomized range finder (rsvd.cu), both factors wanted.
#include <climits>

#include "grid_sync.cuh"
#include "kernels.h"

namespace ptk {

namespace {

constexpr int GRID_THREADS = 512;
constexpr int GROUP_WARPS = 4;
constexpr int GROUPS = GRID_THREADS / 32 / GROUP_WARPS;    // 4 pairs per CTA at a time (2 task slots)
constexpr int MAX_ITEMS = 1024;

template <typename R>
__device__ __forceinline__ R wsumd(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename R> struct Cx;
// A: the matrix on D's shape; B: the matrix B = R^H of the pivoted QR (on_b); V: the right factor
// (the sweeps are written for a real type R; the path instantiates them in FP64)
template <> struct Cx<double> {
  using T = double2;
  static constexpr double EPS = 1.1102230246251565e-16;
  __device__ static T* A(const BondWork& W) { return W.A; }
  __device__ static T* B(const BondWork& W) { return W.G64; }
  __device__ static T* V(const BondWork& W) { return W.V; }
};

__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void item_shape(const BondWork& W, int* Ma, int* Na) {
  const int mD = W.info[0], nD = W.info[1];
  const bool tr = W.info[2] != 0;
  *Ma = (mD > 0 && nD > 0) ? (tr ? nD : mD) : 0;
  *Na = (mD > 0 && nD > 0) ? (tr ? mD : nD) : 0;
}

}  // namespace

// Sum over the 32 lanes of two values at once (a reduce-scatter butterfly): lane 0 ends with the
// total of a, lane 16 with the total of b; 5 shuffles and 5 adds instead of 10 and 10.
template <typename R>
__device__ __forceinline__ R wsum2(R a, R b, int lane) {
  const bool hi = (lane & 16) != 0;
  R keep = hi ? b : a;
  keep += __shfl_xor_sync(0xffffffffu, hi ? a : b, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
  return keep;
}

// One column pair (i, j) of matrix w, processed by the 4 warps of group grp (rows split across
// them). nrm holds the squared column norms: they are read here and, when the pair rotates,
// updated by the rotation's closed form (or recomputed from the columns where that form cancels),
// so the dot phase only forms gamma = a_i^H a_j.
// Counts a rotation in cnt. Every warp of the group must call it.
template <typename R>
__device__ __forceinline__ void process_pair(typename Cx<R>::T* A, typename Cx<R>::T* V, double* nrm, int Ma,
                                             int Na, int i, int j, double fro, double floor_eps, int grp, int gw,
                                             int lane, R (*s_part)[GROUP_WARPS][4], R (*s_rot)[8], int* cnt_slot,
                                             bool with_v, int* stamp, int g_round, int skip_before, R tol) {
  using C2 = typename Cx<R>::T;
  const R eps = Cx<R>::EPS;
  if (i > j) { const int tt = i; i = j; j = tt; }
  const bool real_pair = j < Na;        // uniform within the group
  if (!real_pair) return;
  const bool leader = gw == 0 && lane == 0;
  R al = 0, be = 0;
  if (leader) {
    al = (R)__ldcg(nrm + i);
    be = (R)__ldcg(nrm + j);
  }
  C2* ai = A + (size_t)i * Ma;
  C2* aj = A + (size_t)j * Ma;
  C2* vi = V + (size_t)i * Na;
  C2* vj = V + (size_t)j * Na;
  const int r0 = gw * 32 + lane;
  // the first RC rows of each lane stay in registers for the rotation (all of them when
  // Ma <= RC * 128); the rest, if any, are read again
  constexpr int RC = 2, STEP = 32 * GROUP_WARPS;
  C2 xs[RC], ys[RC];
  const int si = __ldcg(stamp + i), sj = __ldcg(stamp + j);
  {
    R gr = 0, gi = 0;
#pragma unroll
    for (int k = 0; k < RC; ++k) {
      const int r = r0 + k * STEP;
      if (r < Ma) {
        xs[k] = __ldcg(ai + r);
        ys[k] = __ldcg(aj + r);
        gr = fma(xs[k].x, ys[k].x, fma(xs[k].y, ys[k].y, gr));
        gi = fma(xs[k].x, ys[k].y, fma(-xs[k].y, ys[k].x, gi));
      }
    }
    for (int r = r0 + RC * STEP; r < Ma; r += STEP) {
      const C2 x = __ldcg(ai + r), y = __ldcg(aj + r);
      gr = fma(x.x, y.x, fma(x.y, y.y, gr));
      gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
    }
    // unchanged pair: neither column has rotated since this pair was checked one sweep ago (and
    // found orthogonal, or it would carry that round's stamp), so gamma would come out the same
    if (max(si, sj) < skip_before) return;       // uniform: every lane read the same stamps
    const R part = wsum2(gr, gi, lane);
    if (lane == 0) s_part[grp][gw][0] = part;
    if (lane == 16) s_part[grp][gw][1] = part;
  }
  named_sync(1 + grp, 32 * GROUP_WARPS);
  // one lane turns the partial sums (fixed order) into the rotation and shares it
  if (leader) {
    R flag = 0, c = 1, sv = 0, ser = 0, sei = 0, cer = 1, cei = 0;
    R gr = 0, gi = 0;
#pragma unroll
    for (int k = 0; k < GROUP_WARPS; ++k) {
      gr += s_part[grp][k][0];
      gi += s_part[grp][k][1];
    }
    const R g2 = gr * gr + gi * gi;
    const R fl2 = (R)(floor_eps * floor_eps * fro);
    // rotate unless |gamma| <= tol sqrt(alpha beta), or a column is at the noise floor
    // (|a|^2 <= floor_eps^2 ||A||_F^2: such columns cannot become orthogonal relative to
    // their own norm and carry no information at this precision)
    if (g2 > tol * tol * al * be && g2 > R(0) && fmin(al, be) > fl2) {
      // smaller root of the rotation equation: with q = sqrt(h^2 + 4 g^2) and w = q + |h|,
      // |s| / g = sqrt(2 / (q w)), c = w |s| / (2 g) and t g = 2 g^2 sign(h) / w (two dependent
      // long operations instead of four)
      const R ig = rsqrt(g2), h = be - al, ah = fabs(h);          // ig = 1 / |gamma|
      const R q = sqrt(h * h + R(4) * g2), wq = q + ah;
      const R sgm = rsqrt(R(0.5) * q * wq);
      const R sgn = h >= R(0) ? R(1) : R(-1);
      const R sg = sgn * sgm;                                     // s / |gamma|
      c = R(0.5) * wq * sgm;
      sv = sg * g2 * ig;
      ser = sg * gr;                        // s e^{-i phi}: e = conj(gamma) / |gamma|
      sei = -sg * gi;
      const R cg_ = c * ig;
      cer = cg_ * gr;
      cei = -cg_ * gi;
      __stcg(stamp + i, g_round);
      __stcg(stamp + j, g_round);
      const R tg = sgn * g2 * sgm * sgm * q, al2 = al - tg, be2 = be + tg;
      if (al2 >= R(0.25) * al && be2 >= R(0.25) * be) {
        flag = 1;
        __stcg(nrm + i, (double)al2);
        __stcg(nrm + j, (double)be2);
        atomicAdd(cnt_slot, 1);
      } else {
        flag = 2;
      }
    }
    s_rot[grp][0] = flag;
    s_rot[grp][1] = c;
    s_rot[grp][2] = sv;
    s_rot[grp][3] = ser;
    s_rot[grp][4] = sei;
    s_rot[grp][5] = cer;
    s_rot[grp][6] = cei;
  }
  named_sync(1 + grp, 32 * GROUP_WARPS);
  if (s_rot[grp][0] == R(0)) return;
  const R c = s_rot[grp][1], s = s_rot[grp][2], ser = s_rot[grp][3], sei = s_rot[grp][4];
  const R cer = s_rot[grp][5], cei = s_rot[grp][6];
  const bool renorm = s_rot[grp][0] == R(2);
  R na = 0, nb = 0;
  auto rotate = [&](int r, C2 x, C2 y) {
    C2 nx, ny;
    nx.x = c * x.x - (ser * y.x - sei * y.y);
    nx.y = c * x.y - (ser * y.y + sei * y.x);
    ny.x = s * x.x + (cer * y.x - cei * y.y);
    ny.y = s * x.y + (cer * y.y + cei * y.x);
    __stcg(ai + r, nx);
    __stcg(aj + r, ny);
    if (renorm) {
      na = fma(nx.x, nx.x, fma(nx.y, nx.y, na));
      nb = fma(ny.x, ny.x, fma(ny.y, ny.y, nb));
    }
  };
#pragma unroll
  for (int k = 0; k < RC; ++k) {
    const int r = r0 + k * STEP;
    if (r < Ma) rotate(r, xs[k], ys[k]);
  }
  for (int r = r0 + RC * STEP; r < Ma; r += STEP) rotate(r, __ldcg(ai + r), __ldcg(aj + r));
  for (int r = r0; with_v && r < Na; r += 32 * GROUP_WARPS) {
    const C2 x = __ldcg(vi + r), y = __ldcg(vj + r);
    C2 nx, ny;
    nx.x = c * x.x - (ser * y.x - sei * y.y);
    nx.y = c * x.y - (ser * y.y + sei * y.x);
    ny.x = s * x.x + (cer * y.x - cei * y.y);
    ny.y = s * x.y + (cer * y.y + cei * y.x);
    __stcg(vi + r, nx);
    __stcg(vj + r, ny);
  }
  if (!renorm) return;
  // the rotated columns' norms, recomputed
  const R part = wsum2(na, nb, lane);
  if (lane == 0) s_part[grp][gw][2] = part;
  if (lane == 16) s_part[grp][gw][3] = part;
  named_sync(1 + grp, 32 * GROUP_WARPS);
  if (leader) {
    R sa = 0, sb = 0;
#pragma unroll
    for (int k = 0; k < GROUP_WARPS; ++k) {
      sa += s_part[grp][k][2];
      sb += s_part[grp][k][3];
    }
    __stcg(nrm + i, (double)sa);
    __stcg(nrm + j, (double)sb);
    atomicAdd(cnt_slot, 1);
  }
}

// One-sided Jacobi over all matrices of a layer in FP64: on W.A (or on B = R^H in G64) with V in
// W.V. on_b = 1: the matrix
// is the pivoted QR's B = R^H, Na rows and info[8] columns; on_b = 2: the l x l factor in G64,
// l = info[9]. with_v: accumulate the right factor V
// (from V = I when init_v). finalize: write sigma, the normalised left vectors and the order.
// floor_eps: unit roundoff that sets the noise floor; tol_scale: a pair rotates while
// |a_i^H a_j| > tol_scale * unit roundoff * |a_i| |a_j| (0: the row count m; < 0: 4 sqrt(m), the
// resolution of the dot products themselves, for the FP32 sweeps).
// cnt: [n_work][2] rotation counters; sweeps go to info[sweep_slot].
template <typename R>
__global__ void __launch_bounds__(GRID_THREADS)
    k_jacobi_grid(const BondWork* work, int n_work, int max_sweeps, GridSync gs, int* cnt, int* status,
                  int init_v, int finalize, double floor_eps, int sweep_slot, int on_b, int with_v,
                  double tol_scale) {
  using C2 = typename Cx<R>::T;
  __shared__ int s_Na[MAX_ITEMS];
  __shared__ int s_Ma[MAX_ITEMS];
  __shared__ int s_off[MAX_ITEMS + 1];      // prefix of pair counts of the active items this round
  __shared__ unsigned char s_active[MAX_ITEMS];
  __shared__ C2* s_A[MAX_ITEMS];
  __shared__ C2* s_V[MAX_ITEMS];
  __shared__ R s_part[GROUPS][GROUP_WARPS][4];
  __shared__ R s_rot[GROUPS][8];            // rotate flag, c, s, s e^{-i phi}, c e^{-i phi}
  __shared__ double s_fro[MAX_ITEMS];       // ||A||_F^2 per item (noise floor)
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int grp = wid / GROUP_WARPS, gw = wid % GROUP_WARPS;
  const int slot = grp / 2, sub = grp % 2;               // a task slot = 2 groups = 8 warps
  const int n_slots = gridDim.x * (GROUPS / 2);
  const int my_slot = slot * gridDim.x + blockIdx.x;     // consecutive tasks go to different SMs
  const R eps = Cx<R>::EPS;
  if (n_work > MAX_ITEMS) {
    if (blockIdx.x == 0 && tid == 0) atomicOr(status, ST_CAPACITY);
    return;
  }
  __shared__ int s_Nf[MAX_ITEMS];           // on_b: rows of B (= columns of D); else Na
  for (int w = tid; w < n_work; w += blockDim.x) {
    int Ma, Na;
    item_shape(work[w], &Ma, &Na);
    // on_b = 1: B = R^H of the pivoted QR (G64), Na rows and k = info[8] columns (the QR's rank);
    // on_b = 2: the range finder's small square factor (G64), l = info[9] rows and columns
    const int kq = on_b == 1 ? max(0, min(work[w].info[8], Na)) : (on_b == 2 ? max(0, min(work[w].info[9], Na)) : Na);
    s_Nf[w] = on_b == 2 ? kq : Na;
    s_Na[w] = kq;
    s_Ma[w] = on_b == 1 ? Na : (on_b == 2 ? kq : Ma);
    s_active[w] = kq >= 2;
    s_A[w] = on_b ? Cx<R>::B(work[w]) : Cx<R>::A(work[w]);
    s_V[w] = Cx<R>::V(work[w]);
  }
  __syncthreads();
  // V = I (optional), zero counters, column norms (for the noise floor)
  {
    const int gt = blockIdx.x * blockDim.x + tid, ngt = gridDim.x * blockDim.x;
    for (int w = 0; w < n_work; ++w) {
      const int Na = s_Na[w];
      if (init_v && with_v) {
        C2* V = s_V[w];
        for (size_t idx = gt; idx < (size_t)Na * Na; idx += ngt) {
          C2 v;
          v.x = ((idx % Na) == (idx / Na)) ? R(1) : R(0);
          v.y = R(0);
          __stcg(V + idx, v);
        }
      }
      if (gt == 0) {
        cnt[2 * w] = 0;
        cnt[2 * w + 1] = 0;
      }
      for (int c = gt; c < Na; c += ngt) __stcg(work[w].perm + c, -1);   // rotation stamps (perm is free until the end)
    }
    const int gwarp = wid * gridDim.x + blockIdx.x, ngwarp = gridDim.x * (blockDim.x / 32);
    int base = 0;
    for (int w = 0; w < n_work; ++w) {
      const int Ma = s_Ma[w], Na = s_Na[w];
      for (int c = gwarp - base; c < Na; c += ngwarp) {
        if (c < 0) continue;
        const C2* a = s_A[w] + (size_t)c * Ma;
        double s2 = 0;
        for (int r = lane; r < Ma; r += 32) {
          const C2 x = __ldcg(a + r);
          s2 += (double)x.x * x.x + (double)x.y * x.y;
        }
        s2 = wsumd(s2);
        if (lane == 0) __stcg(work[w].aux + c, s2);
      }
      base = (base + Na) % ngwarp;
    }
  }
  if (!grid_barrier(gs, status)) return;
  // ||A||_F^2 per item, summed in the same fixed order by every CTA
  for (int w = wid; w < n_work; w += blockDim.x / 32) {
    double acc = 0;
    for (int k = lane; k < s_Na[w]; k += 32) acc += __ldcg(work[w].aux + k);
    acc = wsumd(acc);
    if (lane == 0) s_fro[w] = acc;
  }
  __syncthreads();
  int sweep = 0;
  bool any = false;
  for (int w = 0; w < n_work; ++w) any |= s_active[w] != 0;
  // fixed stride of the global round index (every matrix's tournament fits in it), so that a pair
  // that meets in round r of every sweep met one stride earlier, whichever matrices are still active
  int stride = 1;
  for (int w = 0; w < n_work; ++w)
    if (s_Na[w] >= 2) {
      const int nb = (s_Na[w] + 1) / 2, nbp = nb + (nb & 1);
      stride = max(stride, nbp - 1);
    }
  while (any && sweep < max_sweeps) {
    const int par = sweep & 1;
    if (blockIdx.x == 0)
      for (int w = tid; w < n_work; w += blockDim.x) cnt[2 * w + (par ^ 1)] = 0;
    // 2-column blocks: a task pairs two blocks and runs their cross pairs (and, in round 0, the
    // pairs inside each block) in sub-rounds separated by a barrier of the task's 8 warps; the
    // round-robin tournament runs over blocks, so a sweep has half as many grid barriers
    int rounds = 0;
    for (int w = 0; w < n_work; ++w)
      if (s_active[w]) {
        const int nb = (s_Na[w] + 1) / 2, nbp = nb + (nb & 1);
        rounds = max(rounds, nbp - 1);
      }
    for (int round = 0; round < rounds; ++round) {
      const int g_round = sweep * stride + round;    // a pair meets in the same round of every sweep
      if (tid == 0) {
        int o = 0;
        for (int w = 0; w < n_work; ++w) {
          s_off[w] = o;
          const int nb = (s_Na[w] + 1) / 2, nbp = nb + (nb & 1);
          if (s_active[w] && round < nbp - 1) o += nbp / 2;
        }
        s_off[n_work] = o;
      }
      __syncthreads();
      const int total = s_off[n_work];
      for (int t = my_slot; t < total; t += n_slots) {
        int lo = 0, hi = n_work - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_off[mid] <= t) lo = mid;
          else hi = mid - 1;
        }
        const int w = lo;
        const int q = t - s_off[w];
        const int Ma = s_Ma[w], Na = s_Na[w];
        const int nb = (Na + 1) / 2, nbp = nb + (nb & 1);
        int bi, bj;
        if (q == 0) { bi = nbp - 1; bj = round; }
        else { bi = (round + q) % (nbp - 1); bj = (round - q + nbp - 1) % (nbp - 1); }
        const int i0 = 2 * bi, j0 = 2 * bj;
        const int n_sub = round == 0 ? 3 : 2;
        for (int sr = 0; sr < n_sub; ++sr) {
          int i, j;
          if (sr == 0) { i = i0 + sub; j = j0 + sub; }
          else if (sr == 1) { i = i0 + sub; j = j0 + 1 - sub; }
          else { i = sub == 0 ? i0 : j0; j = i + 1; }          // pairs inside each block
          process_pair<R>(s_A[w], s_V[w], work[w].aux, Ma, Na, i, j, s_fro[w], floor_eps, grp, gw, lane, s_part,
                          s_rot, &cnt[2 * w + par], with_v != 0, work[w].perm, g_round,
                          sweep > 0 ? g_round - stride : INT_MIN,
                          (R)((tol_scale > 0 ? tol_scale : (tol_scale < 0 ? 4.0 * sqrt((double)Ma) : (double)Ma)) * eps));
          named_sync(9 + slot, 32 * GROUP_WARPS * 2);
        }
      }
      if (!grid_barrier(gs, status)) return;
    }
    // sweep done: retire converged items (every CTA reads the same counters)
    if (tid == 0)
      for (int w = 0; w < n_work; ++w)
        if (s_active[w] && *(volatile int*)&cnt[2 * w + par] == 0) {
          s_active[w] = 0;
          if (blockIdx.x == 0) work[w].info[sweep_slot] = sweep + 1;
        }
    __syncthreads();
    any = false;
    for (int w = 0; w < n_work; ++w) any |= s_active[w] != 0;
    ++sweep;
    if (!grid_barrier(gs, status)) return;
  }
  // a preconditioning run (no finalize) that reaches its sweep cap is not an error: the FP64 sweeps
  // that follow finish the job (and report their own non-convergence)
  if (any && blockIdx.x == 0 && tid == 0) {
    if (finalize) atomicOr(status, ST_SVD_NOCONV);
    for (int w = 0; w < n_work; ++w)
      if (s_active[w]) work[w].info[sweep_slot] = -sweep;
  }
  if (!finalize) return;
  // singular values: column norms, normalise the columns (left vectors), then rank by sigma
  {
    const int gwarp = wid * gridDim.x + blockIdx.x, ngwarp = gridDim.x * (blockDim.x / 32);
    int base = 0;
    for (int w = 0; w < n_work; ++w) {
      const int Ma = s_Ma[w], Na = s_Na[w];
      for (int c = gwarp - base; c < Na; c += ngwarp) {
        if (c < 0) continue;
        C2* a = s_A[w] + (size_t)c * Ma;
        R s2 = 0;
        for (int r = lane; r < Ma; r += 32) {
          const C2 x = __ldcg(a + r);
          s2 += x.x * x.x + x.y * x.y;
        }
        s2 = wsumd(s2);
        const R sg = sqrt(s2);
        if (lane == 0) __stcg(work[w].sig + c, (double)sg);
        if (sg > R(0)) {
          const R inv = R(1) / sg;
          for (int r = lane; r < Ma; r += 32) {
            C2 x = __ldcg(a + r);
            x.x *= inv;
            x.y *= inv;
            __stcg(a + r, x);
          }
        }
        if (lane == 0 && !(sg == sg)) {
          atomicOr(status, ST_NAN);
          atomicOr(work[w].info + 6, FAULT_SIGMA_NAN);
        }
      }
      base = (base + Na) % ngwarp;
    }
  }
  // on_b: the columns of D beyond the QR's rank have singular value 0 (after the sigma of the
  // k columns above, so the ranking below sees every column)
  if (on_b) {
    const int gt = blockIdx.x * blockDim.x + tid, ngt = gridDim.x * blockDim.x;
    for (int w = 0; w < n_work; ++w)
      for (int c = s_Na[w] + gt; c < s_Nf[w]; c += ngt) __stcg(work[w].sig + c, 0.0);
  }
  if (!grid_barrier(gs, status)) return;
  {
    const int gt = blockIdx.x * blockDim.x + tid, ngt = gridDim.x * blockDim.x;
    for (int w = 0; w < n_work; ++w) {
      const int Na = s_Nf[w];
      const double* sig = work[w].sig;
      for (int c = gt; c < Na; c += ngt) {
        // a NaN ranks as -1 so the ranks stay a permutation (perm indexes columns downstream)
        double sc = __ldcg(sig + c);
        if (!(sc == sc)) sc = -1.0;
        int rk = 0;
        for (int k = 0; k < Na; ++k) {
          double sk = __ldcg(sig + k);
          if (!(sk == sk)) sk = -1.0;
          rk += (sk > sc) || (sk == sc && k < c);
        }
        work[w].perm[rk] = c;
      }
    }
  }
}

int jacobi_grid_blocks() {
  int dev = 0, sms = 0, a = 0, b = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_jacobi_grid<double>, GRID_THREADS, 0);
  (void)b;
  return a >= 1 ? sms : 0;
}

void launch_jacobi_grid(const BondWork* work, int n_work, int blocks, int max_sweeps, unsigned* sync3,
                        int* cnt, int* status, cudaStream_t st, int init_v, int finalize,
                        double floor_eps, int sweep_slot, int on_b, int with_v, double tol_scale) {
  // the barrier's arrival counter and the abort flag start at zero for every launch
  cudaMemsetAsync(sync3, 0, sizeof(unsigned), st);
  cudaMemsetAsync(sync3 + 2, 0, sizeof(unsigned), st);
  GridSync gs{sync3, (int*)(sync3 + 2), GRID_WAIT_LIMIT_CYCLES};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks, 1, 1);
  cfg.blockDim = dim3(GRID_THREADS, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_jacobi_grid<double>, work, n_work, max_sweeps, gs, cnt, status, init_v, finalize,
                     floor_eps, sweep_slot, on_b, with_v, tol_scale);
}

}  // namespace ptk
