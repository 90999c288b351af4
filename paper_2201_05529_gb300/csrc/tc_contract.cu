// The fast path's two remaining dense contractions on the tensor cores, each as the sliced BF16
// GEMM of tc_zgemm.cu (six exact slices, FP32 accumulation, FP64 result), between a gather or
// plan kernel and a scatter kernel that put the tensors into and out of GEMM shape.
//
// 1. PT site contraction (App. A.2, the site layer):
//
//   Gamma'[l, p', b, r] = sum_{a, p} Gamma[l, p, a, r] P~[a, p, p', b]
//
// is, for every site, one complex GEMM over all (l, r) pairs:
//
//   X[(l, r), (a, p)] = Gamma[l, p, a, r]                  gather (column-major, ld chi_l chi_r)
//   Y = X opB(P~),  opB(P~)[(a, p), (p', b)] = P~[a, p, p', b]
//   Gamma'[l, p', b, r] = Y[(l, r), (p', b)]                scatter
//
// P~ is read in place: stored [a][p][p'][b], it is the transpose of a column-major
// (4 kappa_out) x (4 kappa_in) matrix with leading dimension 4 kappa_out. One item per site of every
// chain, so the whole site layer is one GEMM launch. X lives in the site's second Gamma buffer, Y in
// a per-site scratch; the scatter writes Gamma' into the second buffer, which k_site_swap then makes
// current, as on the FP64 path.
//
// 2. Gamma recovery after the truncated SVD D = U S V^H (App. A.2, the last step of a bond update):
//
//   Gamma_L[l, p', a, c]   = lambda_l^-1 sum_u Q_L[(l, a), u] U[(u, p'), c]
//   Gamma_R[c, q', b, r]   = lambda_r^-1 conj(sum_v Q_R^H[(b, r), v] V[(q', v), c])
//
// with Q_L (m_L x r_L) and Q_R^H (n_R x r_R) the explicit factors of the outer QR / LQ. Per bond two
// GEMM items: C_L = Q_L opB(U) and C_R = Q_R^H opB(V), the singular vectors read in place through a
// column map (U's rows (u, p') are p'-minor: opB = T with leading dimension 4; V's rows (q', v) are
// v-minor: opB = N with leading dimension 1), the products in the bond's Householder scratch, then
// the scatter applies lambda^-1 and the conjugation. A side without an outer reduction (r = m) reads
// its vectors directly, as k_recover does.
#include "kernels.h"

namespace ptk {

// one thread per site: live dims of this step into the site's GEMM item (M = 0 skips the site)
__global__ void k_site_tc_plan(Tables T, const SiteWork* work, int n_work, ZGemmItem* items) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_work) return;
  const int s = work[w].site, m = work[w].mpo, lam = work[w].lam;
  ZGemmItem& it = items[w];
  it.M = it.N = it.K = 0;
  const int k = *T.step;
  if (k >= T.mpo_K[m]) {
    atomicOr(T.status, ST_PT_RANGE);
    return;
  }
  const int* kap = T.mpo_kappa + T.mpo_kappa_off[m];
  const int ka = kap[k], kb = kap[k + 1];
  const int chl = T.lam_chi[lam], chr = T.lam_chi[lam + 1];
  const size_t tot_in = (size_t)chl * 4 * ka * chr, tot_out = (size_t)chl * 4 * kb * chr;
  if (T.site_kappa[s] != ka || tot_in > T.site_cap[s] || tot_out > T.site_cap[s] ||
      (size_t)chl * chr > (size_t)it.cap_m || 4 * ka > it.cap_k || 4 * kb > it.cap_n) {
    atomicOr(T.status, ST_CAPACITY);
    return;
  }
  const int M = chl * chr;
  it.A = T.site_alt[s];
  it.lda = M;
  it.B = T.mpo_P[T.mpo_P_off[m] + k];
  it.ldb = 4 * kb;
  it.ldc = M;
  it.M = M;
  it.N = 4 * kb;
  it.K = 4 * ka;
}

// X[(l, r), (a, p)] = Gamma[l, p, a, r] into the second buffer; grid (x: elements, y: sites)
__global__ void k_site_tc_gather(Tables T, const SiteWork* work, int n_work, const ZGemmItem* items) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const ZGemmItem& it = items[w];
  if (it.M <= 0) return;
  const int s = work[w].site, lam = work[w].lam;
  const int chr = T.lam_chi[lam + 1], ka = it.K / 4, M = it.M;
  const double2* G = T.site_gam[s];
  double2* X = T.site_alt[s];
  const size_t total = (size_t)M * it.K;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    // idx walks Gamma in storage order [l][p][a][r]: reads and writes both run along r
    const int r = (int)(idx % chr);
    size_t t = idx / chr;
    const int a = (int)(t % ka);
    t /= ka;
    const int p = (int)(t % 4);
    const int l = (int)(t / 4);
    X[(size_t)l * chr + r + (size_t)(a * 4 + p) * M] = G[idx];
  }
}

// Gamma'[l, p', b, r] = Y[(l, r), (p', b)] into the second buffer; grid (x: elements, y: sites)
__global__ void k_site_tc_scatter(Tables T, const SiteWork* work, int n_work, const ZGemmItem* items) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const ZGemmItem& it = items[w];
  if (it.M <= 0) return;
  const int s = work[w].site, lam = work[w].lam;
  const int chr = T.lam_chi[lam + 1], kb = it.N / 4, M = it.M;
  const double2* Y = it.C;
  double2* O = T.site_alt[s];
  const size_t total = (size_t)M * it.N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % chr);
    size_t t = idx / chr;
    const int b = (int)(t % kb);
    t /= kb;
    const int q = (int)(t % 4);
    const int l = (int)(t / 4);
    O[idx] = Y[(size_t)l * chr + r + (size_t)(q * kb + b) * M];
  }
}

// the live shape of a bond's recovery (after the truncation: chi is the new centre bond)
struct RecDims {
  int chl, chi, chr, kL, kR, rL, rR, mL, nR, Ma, Na;
  bool qrL, lqR, tr;
};

__device__ __forceinline__ bool rec_dims(const Tables& T, const BondWork& W, RecDims* d) {
  const int mD = W.info[0], nD = W.info[1];
  if (mD <= 0 || nD <= 0) return false;
  const int sL = W.site_l, BL = W.lam_l;
  d->chl = T.lam_chi[BL];
  d->chi = T.lam_chi[BL + 1];
  d->chr = T.lam_chi[BL + 2];
  d->kL = T.site_kappa[sL];
  d->kR = T.site_kappa[sL + 1];
  d->rL = mD / 4;
  d->rR = nD / 4;
  d->mL = d->chl * d->kL;
  d->nR = d->kR * d->chr;
  d->qrL = d->mL != d->rL;
  d->lqR = d->nR != d->rR;
  d->tr = W.info[2] != 0;
  d->Ma = d->tr ? nD : mD;
  d->Na = d->tr ? mD : nD;
  return true;
}

// one block per bond: the two GEMM items (2w: left, 2w + 1: right) and their column maps
__global__ void k_recover_tc_plan(Tables T, const BondWork* work, int n_work, ZGemmItem* items, int* const* bcols) {
  const int w = blockIdx.x;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  ZGemmItem& iL = items[2 * w];
  ZGemmItem& iR = items[2 * w + 1];
  RecDims d;
  if (!rec_dims(T, W, &d)) {
    if (threadIdx.x == 0) iL.M = iL.N = iL.K = iR.M = iR.N = iR.K = 0;
    return;
  }
  const bool doL = d.qrL && d.chi > 0, doR = d.lqR && d.chi > 0;
  int* bL = bcols[w];
  int* bR = bL + W.nL_cap;
  // U[row, c] and V[row, c] of D = U S V^H (the fast path's kept vectors are in order: perm = identity)
  const double2* Ub = d.tr ? W.V : W.A;
  const double2* Vb = d.tr ? W.A : W.V;
  const int ldU = d.tr ? d.Na : d.Ma, ldV = d.tr ? d.Ma : d.Na;
  for (int n = threadIdx.x; n < 4 * d.chi; n += blockDim.x) {
    const int c = n >> 2, p = n & 3;
    if (doL) bL[n] = p + c * ldU;              // opB(U)[u, (c, p')] = U[4 u + p', c]
    if (doR) bR[n] = p * d.rR + c * ldV;       // opB(V)[v, (c, q')] = V[q' r_R + v, c]
  }
  if (threadIdx.x != 0) return;
  iL.M = iL.N = iL.K = 0;
  iR.M = iR.N = iR.K = 0;
  if (doL && d.mL <= iL.cap_m && d.rL <= iL.cap_k && 4 * d.chi <= iL.cap_n) {
    iL.A = W.QL;
    iL.lda = d.mL;
    iL.B = Ub;
    iL.ldb = 4;
    iL.ldc = d.mL;
    iL.M = d.mL;
    iL.N = 4 * d.chi;
    iL.K = d.rL;
  }
  if (doR && d.nR <= iR.cap_m && d.rR <= iR.cap_k && 4 * d.chi <= iR.cap_n) {
    iR.A = W.QR;
    iR.lda = d.nR;
    iR.B = Vb;
    iR.ldb = 1;
    iR.ldc = d.nR;
    iR.M = d.nR;
    iR.N = 4 * d.chi;
    iR.K = d.rR;
  }
}

// Gamma_L and Gamma_R from the products (or straight from U, V where a side has no reduction);
// grid (x: elements, y: bonds)
__global__ void k_recover_tc_scatter(Tables T, const BondWork* work, int n_work, const ZGemmItem* items) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  RecDims d;
  if (!rec_dims(T, W, &d)) return;
  const int sL = W.site_l, sR = sL + 1, BL = W.lam_l, BR = BL + 2;
  const int chi = d.chi, chl = d.chl, chr = d.chr, kL = d.kL, kR = d.kR;
  const size_t totL = (size_t)chl * 4 * kL * chi, totR = (size_t)chi * 4 * kR * chr;
  if (totL > T.site_cap[sL] || totR > T.site_cap[sR]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(T.status, ST_CAPACITY);
    return;
  }
  const ZGemmItem& iL = items[2 * w];
  const ZGemmItem& iR = items[2 * w + 1];
  if (chi > 0 && ((d.qrL && iL.M == 0) || (d.lqR && iR.M == 0))) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(T.status, ST_CAPACITY);
    return;
  }
  const double* lamL = T.lam_ptr[BL];
  const double* lamR = T.lam_ptr[BR];
  double2* GL = T.site_gam[sL];
  double2* GR = T.site_gam[sR];
  const double2* Ub = d.tr ? W.V : W.A;
  const double2* Vb = d.tr ? W.A : W.V;
  const int ldU = d.tr ? d.Na : d.Ma, ldV = d.tr ? d.Ma : d.Na;
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
      const double2 v = d.qrL ? iL.C[row + (size_t)(c * 4 + pp) * d.mL] : Ub[row * 4 + pp + (size_t)c * ldU];
      GL[idx] = cscale(v, 1.0 / lamL[l]);
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
      const double2 v = d.lqR ? iR.C[colR + (size_t)(c * 4 + qq) * d.nR] : Vb[qq * d.rR + colR + (size_t)c * ldV];
      GR[j] = cscale(cconj(v), 1.0 / lamR[r]);
    }
  }
}

void launch_recover_tc(const Tables& T, const BondWork* work, int n_work, ZGemmItem* items, int* const* bcols,
                       int gx, int tile_cap, int m_cap_max, int n_cap_max, cudaStream_t st) {
  if (n_work <= 0) return;
  k_recover_tc_plan<<<n_work, 128, 0, st>>>(T, work, n_work, items, bcols);
  launch_zgemm(items, 2 * n_work, tile_cap, m_cap_max, n_cap_max, T.status, st);
  k_recover_tc_scatter<<<dim3(gx, n_work), 256, 0, st>>>(T, work, n_work, items);
}

void launch_site_tc(const Tables& T, const SiteWork* work, int n_work, ZGemmItem* items, int gx, int tile_cap,
                    int m_cap_max, int n_cap_max, cudaStream_t st) {
  if (n_work <= 0) return;
  k_site_tc_plan<<<(n_work + 127) / 128, 128, 0, st>>>(T, work, n_work, items);
  k_site_tc_gather<<<dim3(gx, n_work), 256, 0, st>>>(T, work, n_work, items);
  launch_zgemm(items, n_work, tile_cap, m_cap_max, n_cap_max, T.status, st);
  k_site_tc_scatter<<<dim3(gx, n_work), 256, 0, st>>>(T, work, n_work, items);
}

}  // namespace ptk
