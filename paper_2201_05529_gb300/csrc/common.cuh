// Shared device-side definitions of the PT-TEBD engine (tables, work items, complex helpers).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PT_DEV __device__ __forceinline__

// ---------------------------------------------------------------- complex arithmetic (FP64)
PT_DEV double2 cmk(double r, double i) { return make_double2(r, i); }
PT_DEV double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
PT_DEV double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
PT_DEV double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
PT_DEV double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
PT_DEV double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// acc += a * b
PT_DEV double2 cfma(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc += conj(a) * b
PT_DEV double2 cfma_conj(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
PT_DEV double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// counter-based hash -> a value in (-1, 1): a 64-bit finaliser of the counter (no state, the same
// value for the same counter on every launch)
PT_DEV double hash_unit(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdULL;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ULL;
  x ^= x >> 33;
  return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// ---------------------------------------------------------------- device status word codes
enum : int {
  ST_OK = 0,
  ST_CAPACITY = 1,
  ST_SVD_NOCONV = 2,
  ST_NAN = 4,
  ST_PT_RANGE = 8,
  ST_TIMEOUT = 16,
};

// per-update fault flags of one bond (info[6], cleared by the layer's first kernel; the bond log
// keeps them): which check raised ST_NAN for that bond
enum : int {
  FAULT_D_NONFINITE = 1,      // theta + gate produced a NaN or an infinity (the SVD was skipped)
  FAULT_SIGMA_NAN = 2,        // a singular value came out NaN
  FAULT_ZERO_NORM = 4,        // the kept singular values have norm zero or NaN at the truncation
};

// ---------------------------------------------------------------- engine tables (device)
// Global site index s, global bond (lambda) index B. Chain c owns sites
// [site0[c], site0[c] + N[c]) and lambdas [lam0[c], lam0[c] + N[c] + 1).
struct Tables {
  double2** site_gam;      // [n_sites] current Gamma buffer, layout [chi_l][4][kappa][chi_r]
  double2** site_alt;      // [n_sites] second buffer (PT contraction writes here, then swap)
  int* site_kappa;         // [n_sites] live kappa
  int* site_mpo;           // [n_sites] PT-MPO index or -1
  size_t* site_cap;        // [n_sites] capacity of each Gamma buffer (complex elements)
  double** lam_ptr;        // [n_lams] lambda buffers
  int* lam_chi;            // [n_lams] live chi
  int* lam_cap;            // [n_lams] capacity
  double* lam_lognorm;     // [n_lams] accumulated log of the norms removed at that bond
  int* chain_site0;
  int* chain_lam0;
  int* chain_N;
  // PT-MPOs (local propagators already fused)
  int* mpo_K;              // [n_mpos]
  int* mpo_kappa_off;      // [n_mpos] offset into mpo_kappa (K+1 entries each)
  int* mpo_kappa;
  int* mpo_P_off;          // [n_mpos] offset into mpo_P (K pointers each)
  const double2** mpo_P;   // P^(k+1)[kappa_k][4][4][kappa_{k+1}]
  int* mpo_cap_off;        // [n_mpos] offset into mpo_cap (K+1 pointers each)
  double2** mpo_cap;       // C^(k)[kappa_k]
  int* step;               // [1] completed steps
  int* status;             // [1] device status word (ST_* bits)
};

// One two-site bond update (App. A.2) with its private scratch.
struct BondWork {
  int chain;
  int site_l;              // global index of the left site
  int lam_l;               // global lambda index of the bond left of site_l
  int pad;
  const double2* gate;     // 16x16 row-major
  double2* QL;             // [mL_cap * nL_cap]  B_L (col-major) -> Q_L
  double2* RL;             // [nL_cap * nL_cap]  R_L (col-major, upper triangle)
  double2* QR;             // [nR_cap * mR_cap]  B_R^H (col-major) -> Q_R^H
  double2* LR;             // [mR_cap * mR_cap]  R of B_R^H (col-major)
  double2* HH;             // Householder vectors, max(mL*nL, nR*mR)
  double2* A;              // [mD_cap * nD_cap]  D (or D^H) col-major, becomes U (or V)
  double2* V;              // [k_cap * k_cap]    right factor of the one-sided Jacobi
  double* sig;             // [max(k_cap, mR_cap)] singular values (unsorted); B_R^H reflector scalars
  double* aux;             // [max(k_cap, nL_cap)] column norms scratch; B_L reflector scalars
  int* perm;               // [k_cap] perm[rank] = column
  void* TA;                // fast path: packed split planes of the theta operands (tc_theta.cu)
  void* TB;
  double2* G64;            // [k_cap^2] B = R^H of the pivoted QR; fast path: the range finder's l x l factor
  double2* Y64;            // [max(mD,nD)_cap * k_cap] QR workspace / product scratch
  int* qperm;              // [k_cap] column permutation of the pivoted QR
  int* info;               // [16] per-item: 0 mD, 1 nD, 2 transposed, 3 sweeps, 4-5 rotation counters,
                           // 6 fault flags of the update (FAULT_*), 7 NaN flag of theta, 8 rank k of
                           // the pivoted QR, 9 the range finder's width l, 10-11 the update's
                           // discarded weight (a double), 12-13 ||D||_F^2 (a double, fast path)
  // fast path (randomized truncated SVD, rsvd.cu): l <= L_cap columns, rows <= rs_mx
  double2* RY;             // [rs_mx * L_cap]  Y = D Omega, then Q
  double2* RZ;             // [k_cap * L_cap]  Z = D^H Q, then Qz / Qb
  double2* RH;             // [rs_mx * L_cap]  Householder vectors
  double2* RR;             // [L_cap * L_cap]  discarded triangular factors
  double* Rtau;            // [L_cap]
  unsigned char* ZA;       // packed operands of the sliced tensor-core GEMMs (ZA: D or Q as A)
  unsigned char* ZB;
  unsigned char* ZA2;      // D^H as the A operand, packed once per bond update
  int mL_cap, nL_cap, mR_cap, nR_cap, mD_cap, nD_cap, k_cap, pad2;
  int rs_mx, L_cap;        // max(mD_cap, nD_cap) and the range finder's capacity (0: no fast path)
};

struct SiteWork {
  int site;                // global site index
  int mpo;                 // PT-MPO index
  int lam;                 // global lambda index of the bond left of the site
  int pad;
};

// ---------------------------------------------------------------- live dims of one bond update
// B_L = [(l,a),(p,c)] is mL x nL, B_R = [(c,q),(b,r)] is mR x nR; the QR (LQ) reduction runs when
// B_L (B_R) is taller (wider) than its inner dimension; D is mD x nD = 4 rL x 4 rR.
struct BondDims {
  int sL, sR, BL, BC, BR;
  int chl, chc, chr, kL, kR;
  int mL, nL, mR, nR;
  bool qrL, lqR;
  int rL, rR, mD, nD;
};

PT_DEV BondDims bond_dims(const Tables& T, const BondWork& W) {
  BondDims d;
  d.sL = W.site_l; d.sR = W.site_l + 1;
  d.BL = W.lam_l; d.BC = W.lam_l + 1; d.BR = W.lam_l + 2;
  d.chl = T.lam_chi[d.BL]; d.chc = T.lam_chi[d.BC]; d.chr = T.lam_chi[d.BR];
  d.kL = T.site_kappa[d.sL]; d.kR = T.site_kappa[d.sR];
  d.mL = d.chl * d.kL; d.nL = 4 * d.chc;
  d.mR = 4 * d.chc; d.nR = d.kR * d.chr;
  d.qrL = d.mL > d.nL;
  d.lqR = d.nR > d.mR;
  d.rL = d.qrL ? d.nL : d.mL;
  d.rR = d.lqR ? d.mR : d.nR;
  d.mD = 4 * d.rL; d.nD = 4 * d.rR;
  return d;
}

PT_DEV bool bond_fits(const BondDims& d, const BondWork& W) {
  return d.mL <= W.mL_cap && d.nL <= W.nL_cap && d.mR <= W.mR_cap && d.nR <= W.nR_cap &&
         d.mD <= W.mD_cap && d.nD <= W.nD_cap;
}
