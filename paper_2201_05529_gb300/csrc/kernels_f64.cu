// FP64 kernels of the PT-TEBD step (arXiv:2201.05529, App. A.2-A.4).
//
// Every kernel reads the live bond and augmented dimensions from device memory, so one step can
// be captured once as a CUDA graph and replayed while truncation changes chi on the device.
// Gamma buffers are compact: Gamma_n[chi_l][4][kappa][chi_r] with the live dims.
#include "kernels.h"
#include <math.h>

namespace ptk {

PT_DEV size_t gidx(int l, int p, int a, int r, int kap, int chr) {
  return (((size_t)l * 4 + p) * kap + a) * chr + r;
}

PT_DEV double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum; every thread gets the total. `red` holds >= 32 doubles.
PT_DEV double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double out = red[0];
  __syncthreads();
  return out;
}

// ------------------------------------------------------------------ K1: PT site contraction
// App. A.2: Gamma'[l,p',b,r] = sum_{a,p} Gamma[l,p,a,r] P^(k)[a,p,p',b] with k = step+1.
__global__ void k_site_contract(Tables T, const SiteWork* work, int n_work) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const int s = work[w].site, m = work[w].mpo, lam = work[w].lam;
  const int k = *T.step;
  if (k >= T.mpo_K[m]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(T.status, ST_PT_RANGE);
    return;
  }
  const int* kap = T.mpo_kappa + T.mpo_kappa_off[m];
  const int ka = kap[k], kb = kap[k + 1];
  const double2* P = T.mpo_P[T.mpo_P_off[m] + k];
  const int chl = T.lam_chi[lam], chr = T.lam_chi[lam + 1];
  const size_t total = (size_t)chl * 4 * kb * chr;
  if (T.site_kappa[s] != ka || total > T.site_cap[s]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(T.status, ST_CAPACITY);
    return;
  }
  const double2* G = T.site_gam[s];
  double2* O = T.site_alt[s];
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % chr);
    size_t t = idx / chr;
    const int b = (int)(t % kb);
    t /= kb;
    const int q = (int)(t % 4);
    const int l = (int)(t / 4);
    double2 acc = cmk(0, 0);
    for (int a = 0; a < ka; ++a)
#pragma unroll
      for (int p = 0; p < 4; ++p)
        acc = cfma(G[gidx(l, p, a, r, ka, chr)], P[((size_t)(a * 4 + p) * 4 + q) * kb + b], acc);
    O[idx] = acc;
  }
}

// Swap the contracted buffer in and set the new augmented dimension.
__global__ void k_site_swap(Tables T, const SiteWork* work, int n_work) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_work) return;
  const int s = work[w].site, m = work[w].mpo;
  const int k = *T.step;
  if (k >= T.mpo_K[m]) return;
  double2* t = T.site_gam[s];
  T.site_gam[s] = T.site_alt[s];
  T.site_alt[s] = t;
  T.site_kappa[s] = T.mpo_kappa[T.mpo_kappa_off[m] + k + 1];
}

// ------------------------------------------------------------------ K2a: B_L and B_R^H
// App. A.2: B_L = lambda_{n-1} Gamma_n as [(l,a),(p,c)], B_R = Gamma_{n+1} lambda_{n+1} as
// [(c,q),(b,r)]. B_L is stored column-major in QL; B_R^H column-major in QR.
__global__ void k_build_blocks(Tables T, const BondWork* work, int n_work) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  const BondDims d = bond_dims(T, W);
  if (blockIdx.x == 0 && threadIdx.x == 0) W.info[6] = 0;   // this update's fault flags
  if (!bond_fits(d, W)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(T.status, ST_CAPACITY);
    return;
  }
  const double2* GL = T.site_gam[d.sL];
  const double2* GR = T.site_gam[d.sR];
  const double* lamL = T.lam_ptr[d.BL];
  const double* lamR = T.lam_ptr[d.BR];
  const size_t totL = (size_t)d.mL * d.nL, totR = (size_t)d.nR * d.mR;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < totL + totR;
       idx += (size_t)gridDim.x * blockDim.x) {
    if (idx < totL) {
      const int row = (int)(idx % d.mL), col = (int)(idx / d.mL);
      const int l = row / d.kL, a = row % d.kL, p = col / d.chc, c = col % d.chc;
      W.QL[idx] = cscale(GL[gidx(l, p, a, c, d.kL, d.chc)], lamL[l]);
    } else {
      const size_t j = idx - totL;
      const int row = (int)(j % d.nR), col = (int)(j / d.nR);
      const int b = row / d.chr, r = row % d.chr, c = col / 4, q = col % 4;
      W.QR[j] = cscale(cconj(GR[gidx(c, q, b, r, d.kR, d.chr)]), lamR[r]);
    }
  }
}

// ------------------------------------------------------------------ K2b: Householder QR
// In place on a column-major M x Nc matrix (M > Nc): reflectors P_j = I - tau_j u_j u_j^H
// (u_j[j] = 1, Hermitian, unitary) with P_{Nc-1}..P_0 A = [R; 0]. R is copied out (col-major
// Nc x Nc) and A is overwritten by the explicit Q = P_0 .. P_{Nc-1} [I; 0].
constexpr int QR_THREADS = 512;
constexpr int QR_MAX_N = 2048;

PT_DEV void householder_qr(double2* A, int M, int Nc, double2* R, double2* H, double* tau,
                           double* red) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < Nc; ++j) {
    double2* x = A + (size_t)j * M;
    double part = 0.0;
    for (int i = j + tid; i < M; i += blockDim.x) part += cabs2(x[i]);
    const double nrm2 = block_sum(part, red);
    const double2 alpha = x[j];
    const double aabs = sqrt(cabs2(alpha));
    const double nrm = sqrt(nrm2);
    double t = 0.0;
    double2 uj = cmk(1, 0), beta = alpha;
    if (nrm > 0.0) {
      const double2 ph = aabs > 0.0 ? cscale(alpha, 1.0 / aabs) : cmk(1, 0);
      beta = cscale(ph, -nrm);
      uj = cscale(ph, aabs + nrm);                // u_j = alpha - beta
      const double u2 = nrm2 - aabs * aabs + cabs2(uj);
      t = 2.0 * cabs2(uj) / u2;
    }
    // u' = x / u_j stored in H (col j); H[j] = 1
    const double inv = 1.0 / cabs2(uj);
    const double2 ujinv = cscale(cconj(uj), inv);
    double2* u = H + (size_t)j * M;
    for (int i = j + tid; i < M; i += blockDim.x) {
      u[i] = (i == j) ? cmk(1, 0) : (nrm > 0.0 ? cmul(x[i], ujinv) : cmk(0, 0));
    }
    if (tid == 0) tau[j] = t;
    __syncthreads();
    for (int i = j + tid; i < M; i += blockDim.x) x[i] = (i == j) ? beta : cmk(0, 0);
    // trailing columns: y -= tau u (u^H y)
    if (t != 0.0) {
      for (int k = j + 1 + wid; k < Nc; k += nw) {
        double2* y = A + (size_t)k * M;
        double2 s = cmk(0, 0);
        for (int i = j + lane; i < M; i += 32) s = cfma_conj(u[i], y[i], s);
        s.x = warp_sum(s.x);
        s.y = warp_sum(s.y);
        const double2 ts = cscale(s, t);
        for (int i = j + lane; i < M; i += 32) y[i] = csub(y[i], cmul(u[i], ts));
      }
    }
    __syncthreads();
  }
  // R out (upper triangle, col-major Nc x Nc)
  for (size_t idx = tid; idx < (size_t)Nc * Nc; idx += blockDim.x) {
    const int r = (int)(idx % Nc), c = (int)(idx / Nc);
    R[idx] = (r <= c) ? A[(size_t)c * M + r] : cmk(0, 0);
  }
  __syncthreads();
  // Q = P_0 ... P_{Nc-1} [I;0]
  for (size_t idx = tid; idx < (size_t)M * Nc; idx += blockDim.x) {
    const int r = (int)(idx % M), c = (int)(idx / M);
    A[idx] = (r == c) ? cmk(1, 0) : cmk(0, 0);
  }
  __syncthreads();
  for (int j = Nc - 1; j >= 0; --j) {
    const double t = tau[j];
    if (t != 0.0) {
      const double2* u = H + (size_t)j * M;
      for (int k = j + wid; k < Nc; k += nw) {
        double2* y = A + (size_t)k * M;
        double2 s = cmk(0, 0);
        for (int i = j + lane; i < M; i += 32) s = cfma_conj(u[i], y[i], s);
        s.x = warp_sum(s.x);
        s.y = warp_sum(s.y);
        const double2 ts = cscale(s, t);
        for (int i = j + lane; i < M; i += 32) y[i] = csub(y[i], cmul(u[i], ts));
      }
    }
    __syncthreads();
  }
}

// blockIdx.x = work item, blockIdx.y = side (0: QR of B_L, 1: QR of B_R^H, i.e. LQ of B_R)
__global__ void __launch_bounds__(QR_THREADS) k_householder(Tables T, const BondWork* work, int n_work) {
  __shared__ double red[32];
  __shared__ double tau[QR_MAX_N];
  const int w = blockIdx.x;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  const BondDims d = bond_dims(T, W);
  if (!bond_fits(d, W)) return;
  if (blockIdx.y == 0) {
    if (!d.qrL || d.nL > QR_MAX_N) return;
    householder_qr(W.QL, d.mL, d.nL, W.RL, W.HH, tau, red);
  } else {
    if (!d.lqR || d.mR > QR_MAX_N) return;
    householder_qr(W.QR, d.nR, d.mR, W.LR, W.HH + (size_t)W.mL_cap * W.nL_cap, tau, red);
  }
}

// ------------------------------------------------------------------ K3: theta + gate
// App. A.2: D[(u,p'),(q',v)] = sum_{pq} G[p'q',pq] sum_c R_L[u,(p,c)] lambda_c L_R[(c,q),v].
// D (m >= n) or D^H (m < n) is written column-major into W.A for the one-sided Jacobi.
__global__ void k_theta_gate(Tables T, const BondWork* work, int n_work) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  const BondDims d = bond_dims(T, W);
  if (!bond_fits(d, W)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) W.info[0] = W.info[1] = 0;   // downstream stages skip
    return;
  }
  const bool tr = d.mD < d.nD;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    W.info[0] = d.mD;
    W.info[1] = d.nD;
    W.info[2] = tr ? 1 : 0;
  }
  const double2* RLp = d.qrL ? W.RL : W.QL;
  const int ldRL = d.qrL ? d.nL : d.mL;
  const double2* LRp = d.lqR ? W.LR : W.QR;       // L_R(row, v) = conj(LRp[v + row * ldLR])
  const int ldLR = d.lqR ? d.mR : d.nR;
  const double* lamC = T.lam_ptr[d.BC];
  __shared__ double2 g[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) g[i] = W.gate[i];
  __syncthreads();
  const int total = d.rL * d.rR;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int u = idx / d.rR, v = idx % d.rR;
    double2 th[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) th[i] = cmk(0, 0);
    for (int c = 0; c < d.chc; ++c) {
      const double lc = lamC[c];
      double2 rl[4], lr[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) rl[p] = cscale(RLp[u + (size_t)(p * d.chc + c) * ldRL], lc);
#pragma unroll
      for (int q = 0; q < 4; ++q) lr[q] = cconj(LRp[v + (size_t)(c * 4 + q) * ldLR]);
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) th[p * 4 + q] = cfma(rl[p], lr[q], th[p * 4 + q]);
    }
#pragma unroll 1
    for (int pp = 0; pp < 4; ++pp) {
#pragma unroll 1
      for (int qq = 0; qq < 4; ++qq) {
        double2 acc = cmk(0, 0);
#pragma unroll
        for (int i = 0; i < 16; ++i) acc = cfma(g[(pp * 4 + qq) * 16 + i], th[i], acc);
        const int row = u * 4 + pp, col = qq * d.rR + v;
        if (!(isfinite(acc.x) && isfinite(acc.y))) W.info[7] = 1;    // k_nan_guard stops this bond
        if (!tr) W.A[row + (size_t)col * d.mD] = acc;
        else W.A[col + (size_t)row * d.nD] = cconj(acc);
      }
    }
  }
}

// ------------------------------------------------------------------ NaN guard before the SVD
// The theta kernels flag a bond whose D holds a NaN or an infinity (info[7]); such a D must not
// reach the SVD (a NaN has no place in a pivot order or a rotation), so the bond is marked empty
// (info[0] = info[1] = 0: the SVD, the truncation and the recovery skip it, the state keeps its
// previous tensors) and the device status records ST_NAN, which the host reports at its next
// synchronising call. One thread per bond; the flag is cleared for the next layer.
__global__ void k_nan_guard(Tables T, const BondWork* work, int n_work) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  if (W.info[7] != 0) {
    W.info[0] = 0;
    W.info[1] = 0;
    W.info[7] = 0;
    W.info[6] |= FAULT_D_NONFINITE;
    atomicOr(T.status, ST_NAN);
  }
}

// ------------------------------------------------------------------ K4: the SVD of D
// The one-sided Jacobi SVD runs as a cluster-parallel kernel (jacobi_cluster.cu).

// ------------------------------------------------------------------ K5: truncation
// App. A.2: the smallest chi with ||discarded||_2 < eps * s_max, capped at chi_max; exact zeros
// dropped; a cut may not split a multiplet (relative gap <= mtol). lambda = kept / ||kept||_2 and
// log||kept||_2 goes into the bond's log-norm accumulator.
PT_DEV int truncation_rank(const double* sig, const int* perm, int n, double eps, int chi_max,
                           double mtol) {
  if (n <= 0) return 1;
  const double smax = sig[perm[0]];
  if (!(smax > 0.0)) return 1;
  const double thr = eps * smax;
  int chi = n;
  double tail2 = 0.0;
  for (int c = n; c >= 1; --c) {
    if (sqrt(tail2) < thr) chi = c;
    else break;
    tail2 += sig[perm[c - 1]] * sig[perm[c - 1]];
  }
  int nz = 0;
  for (int i = 0; i < n; ++i) nz += sig[perm[i]] > 0.0;
  chi = max(1, min(chi, nz));
  auto splits = [&](int c) {
    return c > 0 && c < n && (sig[perm[c - 1]] - sig[perm[c]]) <= mtol * smax;
  };
  if (chi <= chi_max) {
    while (splits(chi) && chi < chi_max && sig[perm[chi]] > 0.0) ++chi;
    if (!splits(chi)) return chi;
  }
  chi = min(chi, chi_max);
  while (chi > 1 && splits(chi)) --chi;
  return chi;
}

__global__ void k_truncate(Tables T, const BondWork* work, int n_work, int chi_max, double eps,
                           double mtol, int rsvd) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  const int mD = W.info[0], nD = W.info[1];
  if (mD <= 0 || nD <= 0) return;
  int n = min(mD, nD);
  if (rsvd) {
    // the fast path's range finder: l computed values; what lies outside its subspace is one
    // lumped value (never kept: chi <= chi_max < l whenever l < n)
    const int l = W.info[9];
    if (l <= 0) return;
    if (l < n) {
      W.sig[l] = sqrt(fmax(0.0, *(const double*)(W.info + 12)));     // ||D - Q Q^H D||_F
      W.perm[l] = l;
      n = l + 1;
    } else {
      n = l;
    }
  }
  const int BC = W.lam_l + 1;
  int chi = truncation_rank(W.sig, W.perm, n, eps, chi_max, mtol);
  if (chi > T.lam_cap[BC]) {
    atomicOr(T.status, ST_CAPACITY);
    chi = T.lam_cap[BC];
  }
  double n2 = 0.0;
  for (int i = 0; i < chi; ++i) n2 += W.sig[W.perm[i]] * W.sig[W.perm[i]];
  const double nrm = sqrt(n2);
  double* lam = T.lam_ptr[BC];
  if (nrm > 0.0 && nrm == nrm) {
    for (int i = 0; i < chi; ++i) lam[i] = W.sig[W.perm[i]] / nrm;
    T.lam_lognorm[BC] += log(nrm);
  } else {
    atomicOr(T.status, ST_NAN);
    W.info[6] |= FAULT_ZERO_NORM;
    for (int i = 0; i < chi; ++i) lam[i] = 0.0;
  }
  T.lam_chi[BC] = chi;
  // discarded weight ||sigma_{>= chi}||_2 / sigma_max of this update, for the bond log
  double tail2 = 0.0;
  for (int i = chi; i < n; ++i) tail2 += W.sig[W.perm[i]] * W.sig[W.perm[i]];
  const double smax = W.sig[W.perm[0]];
  *(double*)(W.info + 10) = smax > 0.0 ? sqrt(tail2) / smax : 0.0;
}

// ------------------------------------------------------------------ bond log
// One record per bond update (one thread per bond of the layer): D's shape, the pivoted QR's rank,
// the Jacobi sweeps, the update's fault flags (FAULT_*), the new bond dimension, the two sites'
// augmented dimensions, and the discarded weight (two ints holding a double). log: [steps][6 layers][nb][BOND_LOG_INTS].
__global__ void k_bond_log(Tables T, const BondWork* work, int n_work, int layer, int* log, int cap_steps,
                           int nb) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_work) return;
  const int k = *T.step;
  if (k >= cap_steps) return;
  const BondWork& W = work[w];
  int* r = log + (((size_t)k * 6 + layer) * nb + w) * BOND_LOG_INTS;
  r[0] = W.info[0];
  r[1] = W.info[1];
  r[2] = W.info[8];
  r[3] = W.info[3];
  r[4] = W.info[6];
  r[5] = T.lam_chi[W.lam_l + 1];
  r[6] = T.site_kappa[W.site_l];
  r[7] = T.site_kappa[W.site_l + 1];
  r[8] = W.info[10];
  r[9] = W.info[11];
}

// ------------------------------------------------------------------ autotuner's synthetic state
__global__ void k_tune_fill(Tables T, int n_sites, int n_lams, unsigned seed) {
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (size_t)gridDim.x * blockDim.x;
  for (int s = 0; s < n_sites; ++s) {
    double2* G = T.site_gam[s];
    const unsigned long long base = ((unsigned long long)seed << 40) ^ ((unsigned long long)s << 28);
    for (size_t i = tid; i < T.site_cap[s]; i += nt)
      G[i] = make_double2(hash_unit(base + 2 * i), hash_unit(base + 2 * i + 1));
  }
  for (int B = 0; B < n_lams; ++B) {
    const int chi = T.lam_chi[B];
    double nrm2 = 0.0;
    for (int i = 0; i < chi; ++i) nrm2 += exp(-i / 4.0);          // sum of the squares below
    for (size_t i = tid; i < (size_t)chi; i += nt) T.lam_ptr[B][i] = exp(-(double)i / 8.0) / sqrt(nrm2);
  }
}

// ------------------------------------------------------------------ K6: Gamma recovery
// App. A.2: Gamma_L = lambda_{n-1}^{-1} Q_L U, Gamma_R = V^H Q_R lambda_{n+1}^{-1}.
__global__ void k_recover(Tables T, const BondWork* work, int n_work) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  const int mD = W.info[0], nD = W.info[1];
  if (mD <= 0 || nD <= 0) return;
  // dims: chi of the centre bond is already the truncated one; recompute the rest
  const int sL = W.site_l, sR = sL + 1, BL = W.lam_l, BC = BL + 1, BR = BL + 2;
  const int chl = T.lam_chi[BL], chi = T.lam_chi[BC], chr = T.lam_chi[BR];
  const int kL = T.site_kappa[sL], kR = T.site_kappa[sR];
  const int rL = mD / 4, rR = nD / 4;
  const int mL = chl * kL, nR = kR * chr;
  const bool qrL = mL != rL;   // rL == mL exactly when no QR was applied
  const bool lqR = nR != rR;
  const bool tr = W.info[2] != 0;
  const int Ma = tr ? nD : mD, Na = tr ? mD : nD;
  const size_t totL = (size_t)chl * 4 * kL * chi, totR = (size_t)chi * 4 * kR * chr;
  if (totL > T.site_cap[sL] || totR > T.site_cap[sR]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(T.status, ST_CAPACITY);
    return;
  }
  const double* lamL = T.lam_ptr[BL];
  const double* lamR = T.lam_ptr[BR];
  double2* GL = T.site_gam[sL];
  double2* GR = T.site_gam[sR];
  // U[row, c] and V[row, c] of D = U S V^H, c = rank
  auto Uel = [&](int row, int c) -> double2 {
    const int col = W.perm[c];
    return tr ? W.V[row + (size_t)col * Na] : W.A[row + (size_t)col * Ma];
  };
  auto Vel = [&](int row, int c) -> double2 {
    const int col = W.perm[c];
    return tr ? W.A[row + (size_t)col * Ma] : W.V[row + (size_t)col * Na];
  };
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < totL + totR;
       idx += (size_t)gridDim.x * blockDim.x) {
    if (idx < totL) {
      // Gamma_L[l][p'][a][c]
      const int c = (int)(idx % chi);
      size_t t = idx / chi;
      const int a = (int)(t % kL);
      t /= kL;
      const int pp = (int)(t % 4);
      const int l = (int)(t / 4);
      const int row = l * kL + a;
      double2 acc;
      if (qrL) {
        acc = cmk(0, 0);
        for (int u = 0; u < rL; ++u) acc = cfma(W.QL[row + (size_t)u * mL], Uel(u * 4 + pp, c), acc);
      } else {
        acc = Uel(row * 4 + pp, c);
      }
      GL[idx] = cscale(acc, 1.0 / lamL[l]);
    } else {
      // Gamma_R[c][q'][b][r]
      const size_t j = idx - totL;
      const int r = (int)(j % chr);
      size_t t = j / chr;
      const int b = (int)(t % kR);
      t /= kR;
      const int qq = (int)(t % 4);
      const int c = (int)(t / 4);
      const int colR = b * chr + r;
      double2 acc;
      if (lqR) {
        // Q_R[v, colR] = conj(Qa[colR + v * nR]), Qa = QR buffer (nR x mR)
        acc = cmk(0, 0);
        for (int v = 0; v < rR; ++v)
          acc = cfma(cconj(Vel(qq * rR + v, c)), cconj(W.QR[colR + (size_t)v * nR]), acc);
      } else {
        acc = cconj(Vel(qq * rR + colR, c));
      }
      GR[j] = cscale(acc, 1.0 / lamR[r]);
    }
  }
}

// ------------------------------------------------------------------ K7: caps
// App. A.3: C^(K) = 1, C^(k-1)[a] = sum_{b,i,o} P^(k)[a,i,o,b] (iota_i / 2) tau_o C^(k)[b] with
// iota = tau = vec(I) = (1,0,0,1). One block per PT-MPO, sequential in k.
__global__ void k_caps(Tables T, int n_mpos) {
  const int m = blockIdx.x;
  if (m >= n_mpos) return;
  const int K = T.mpo_K[m];
  const int* kap = T.mpo_kappa + T.mpo_kappa_off[m];
  double2** C = T.mpo_cap + T.mpo_cap_off[m];
  for (int b = threadIdx.x; b < kap[K]; b += blockDim.x) C[K][b] = cmk(1, 0);
  __syncthreads();
  for (int k = K; k >= 1; --k) {
    const double2* P = T.mpo_P[T.mpo_P_off[m] + k - 1];
    const int ka = kap[k - 1], kb = kap[k];
    for (int a = threadIdx.x; a < ka; a += blockDim.x) {
      double2 acc = cmk(0, 0);
      for (int b = 0; b < kb; ++b) {
        double2 s = cmk(0, 0);
        const int io[2] = {0, 3};
        for (int x = 0; x < 2; ++x)
          for (int y = 0; y < 2; ++y)
            s = cadd(s, P[((size_t)(a * 4 + io[x]) * 4 + io[y]) * kb + b]);
        acc = cfma(s, C[k][b], acc);
      }
      C[k - 1][a] = cscale(acc, 0.5);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ K8: readout
// Contract each augmented leg with its cap C^(k), close Liouville legs with vec(I) except
// vec(O^T) on the measured site, including the lambdas (App. A.3); one block per chain.
// Writes obs[c][n][j] (complex, raw Tr(O rho) times exp(lognorm)) and trace[c].
// M_n[l][p][r] = sum_a Gamma_n[l,p,a,r] C_n^(k)[a]: each site tensor with its augmented leg
// closed by the current cap (App. A.3), for every site of every chain in one launch
// (grid: x over elements, y over chains, z over sites), so that the readout passes below work on
// the small M_n instead of contracting the kappa leg again in each pass.
__global__ void k_observe_m(Tables T, int n_chains, double2* Mbuf, const size_t* moff) {
  const int c = blockIdx.y, n = blockIdx.z;
  if (c >= n_chains || n >= T.chain_N[c]) return;
  const int k = *T.step;
  const int s = T.chain_site0[c] + n, B = T.chain_lam0[c] + n;
  const int chl = T.lam_chi[B], chr = T.lam_chi[B + 1], kap = T.site_kappa[s];
  const double2* G = T.site_gam[s];
  const int m = T.site_mpo[s];
  const double2* capv = m >= 0 ? T.mpo_cap[T.mpo_cap_off[m] + k] : nullptr;
  double2* M = Mbuf + moff[s];
  const size_t tot = (size_t)chl * 4 * chr;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % chr);
    const size_t t = idx / chr;
    const int p = (int)(t % 4), l = (int)(t / 4);
    double2 v = cmk(0, 0);
    for (int a = 0; a < kap; ++a) v = cfma(G[gidx(l, p, a, r, kap, chr)], capv ? capv[a] : cmk(1, 0), v);
    M[idx] = v;
  }
}

__global__ void k_observe(Tables T, int n_chains, const double2* ops, int n_ops, int n_max,
                          double2* obs, double2* trace, double2* Lbuf, double2* Rbuf, int ld,
                          int use_history, const double2* Mbuf, const size_t* moff) {
  const int c = blockIdx.x;
  if (c >= n_chains) return;
  __shared__ double red[32];
  const int k = *T.step;
  const int N = T.chain_N[c], s0 = T.chain_site0[c], B0 = T.chain_lam0[c];
  double2* Lp = Lbuf + (size_t)c * (n_max + 1) * ld;
  double2* Rs = Rbuf + (size_t)c * (n_max + 1) * ld;
  if (use_history) {
    obs += (size_t)k * n_chains * n_max * n_ops;
    trace += (size_t)k * n_chains;
  }
  // M_n[l][p][r] (k_observe_m) at index (l * 4 + p) * chr + r
  auto Mel = [&](int n, int l, int p, int r, int chr) -> double2 {
    return Mbuf[moff[s0 + n] + ((size_t)l * 4 + p) * chr + r];
  };
  // left prefix: Lp[0] = lambda_0; Lp[n+1][r] = lambda_{n+1}[r] sum_l Lp[n][l] V_n[l][r]
  if (threadIdx.x == 0) Lp[0] = cmk(T.lam_ptr[B0][0], 0);
  __syncthreads();
  for (int n = 0; n < N; ++n) {
    const int chl = T.lam_chi[B0 + n], chr = T.lam_chi[B0 + n + 1];
    const double* lr = T.lam_ptr[B0 + n + 1];
    for (int r = threadIdx.x; r < chr; r += blockDim.x) {
      double2 acc = cmk(0, 0);
      for (int l = 0; l < chl; ++l) {
        const double2 v = cadd(Mel(n, l, 0, r, chr), Mel(n, l, 3, r, chr));   // trace of the site
        acc = cfma(Lp[(size_t)n * ld + l], v, acc);
      }
      Lp[(size_t)(n + 1) * ld + r] = cscale(acc, lr[r]);
    }
    __syncthreads();
  }
  // right suffix: Rs[N] = 1; Rs[n][l] = sum_r V_n[l][r] lambda_{n+1}[r] Rs[n+1][r]
  if (threadIdx.x == 0) Rs[(size_t)N * ld] = cmk(1, 0);
  __syncthreads();
  for (int n = N - 1; n >= 0; --n) {
    const int chl = T.lam_chi[B0 + n], chr = T.lam_chi[B0 + n + 1];
    const double* lr = T.lam_ptr[B0 + n + 1];
    for (int l = threadIdx.x; l < chl; l += blockDim.x) {
      double2 acc = cmk(0, 0);
      for (int r = 0; r < chr; ++r) {
        const double2 v = cadd(Mel(n, l, 0, r, chr), Mel(n, l, 3, r, chr));
        acc = cfma(v, cscale(Rs[(size_t)(n + 1) * ld + r], lr[r]), acc);
      }
      Rs[(size_t)n * ld + l] = acc;
    }
    __syncthreads();
  }
  // log-norm (fixed summation order)
  double lognorm = 0.0;
  for (int b = 0; b <= N; ++b) lognorm += T.lam_lognorm[B0 + b];
  const double scale = exp(lognorm);
  if (threadIdx.x == 0) trace[c] = cscale(Lp[(size_t)N * ld], scale);
  // per site and op
  for (int n = 0; n < N; ++n) {
    const int chl = T.lam_chi[B0 + n], chr = T.lam_chi[B0 + n + 1];
    const double* lr = T.lam_ptr[B0 + n + 1];
    for (int j = 0; j < n_ops; ++j) {
      const double2* o = ops + j * 4;
      double2 part = cmk(0, 0);
      for (size_t idx = threadIdx.x; idx < (size_t)chl * chr; idx += blockDim.x) {
        const int l = (int)(idx / chr), r = (int)(idx % chr);
        double2 v = cmk(0, 0);
#pragma unroll
        for (int p = 0; p < 4; ++p) v = cfma(o[p], Mel(n, l, p, r, chr), v);
        const double2 left = Lp[(size_t)n * ld + l];
        const double2 right = cscale(Rs[(size_t)(n + 1) * ld + r], lr[r]);
        part = cfma(cmul(left, v), right, part);
      }
      const double sr = block_sum(part.x, red);
      const double si = block_sum(part.y, red);
      if (threadIdx.x == 0) obs[((size_t)c * n_max + n) * n_ops + j] = cscale(cmk(sr, si), scale);
    }
  }
}

// ------------------------------------------------------------------ K9: local super-operator
// App. A.4: Gamma[l,p,a,r] <- sum_q S[p,q] Gamma[l,q,a,r], S = A (x) I (left) or I (x) A^T (right).
struct Super4 { double2 s[16]; };
__global__ void k_apply_local(Tables T, int site, int lam, Super4 S) {
  const int chl = T.lam_chi[lam], chr = T.lam_chi[lam + 1], kap = T.site_kappa[site];
  double2* G = T.site_gam[site];
  const size_t tot = (size_t)chl * kap * chr;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % chr);
    const size_t t = idx / chr;
    const int a = (int)(t % kap), l = (int)(t / kap);
    double2 x[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) x[p] = G[gidx(l, p, a, r, kap, chr)];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      double2 acc = cmk(0, 0);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc = cfma(S.s[p * 4 + q], x[q], acc);
      G[gidx(l, p, a, r, kap, chr)] = acc;
    }
  }
}

__global__ void k_step_inc(int* step) { *step += 1; }

// ------------------------------------------------------------------ standalone batched SVD
// For the kernel-level entry point: load row-major A_b (m x n) into column-major (or the
// conjugate transpose when m < n); after the cluster Jacobi, write sigma (descending), U, V
// row-major.
__global__ void k_svd_load(const double2* A, int m, int n, int batch, double2* work_A,
                           size_t strideA) {
  const int b = blockIdx.y;
  if (b >= batch) return;
  const bool tr = m < n;
  const int Ma = tr ? n : m;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (size_t)m * n;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    const double2 v = A[(size_t)b * m * n + idx];
    if (!tr) work_A[b * strideA + i + (size_t)j * Ma] = v;
    else work_A[b * strideA + j + (size_t)i * Ma] = cconj(v);
  }
}

__global__ void k_svd_store(const double2* work_A, const double2* work_V, const double* sig,
                            const int* perm, int m, int n, int batch, size_t strideA,
                            size_t strideV, double* sigma_out, double2* U, double2* V) {
  const int b = blockIdx.y;
  if (b >= batch) return;
  const bool tr = m < n;
  const int Ma = tr ? n : m, Na = tr ? m : n, k = Na;
  const double2* WA = work_A + b * strideA;
  const double2* WV = work_V + b * strideV;
  const double* sg = sig + (size_t)b * Na;
  const int* pm = perm + (size_t)b * Na;
  const size_t totU = (size_t)m * k, totV = (size_t)n * k;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < totU + totV + k;
       idx += (size_t)gridDim.x * blockDim.x) {
    if (idx < totU) {
      const int i = (int)(idx / k), c = (int)(idx % k);
      const int col = pm[c];
      U[(size_t)b * totU + idx] = tr ? WV[i + (size_t)col * Na] : WA[i + (size_t)col * Ma];
    } else if (idx < totU + totV) {
      const size_t j = idx - totU;
      const int i = (int)(j / k), c = (int)(j % k);
      const int col = pm[c];
      V[(size_t)b * totV + j] = tr ? WA[i + (size_t)col * Ma] : WV[i + (size_t)col * Na];
    } else {
      const int c = (int)(idx - totU - totV);
      sigma_out[(size_t)b * k + c] = sg[pm[c]];
    }
  }
}

}  // namespace ptk

namespace ptk {
void launch_apply_local(const Tables& T, int site, int lam, const double2* s16, cudaStream_t st) {
  Super4 S;
  for (int i = 0; i < 16; ++i) S.s[i] = s16[i];
  k_apply_local<<<152, 256, 0, st>>>(T, site, lam, S);
}
}  // namespace ptk
