// The fast path's bond SVD as a randomized truncated SVD (App. A.2): the SVD of D only has to
// deliver the chi <= chi_max leading singular triplets and the norm of everything it discards, so
// the fast path finds them in an l-dimensional subspace, l = min(n, chi_max + p), p = 32 extra
// directions (Halko, Martinsson and Tropp's range finder with q = RSVD_POWER power iterations):
//
//   Y  = D Omega,   Q  = qr(Y)          (Omega: n x l, fixed pseudo-random entries)
//   q times:
//   Z  = D^H Q,     Qz = qr(Z)          (a power iteration: sharpens the decay by sigma^2)
//   Y  = D Qz,      Q  = qr(Y)
//   Z  = D^H Q = Qb Rb                  (Z = B^H for B = Q^H D, the l x n projection of D)
//   Rb = Ur S Wr^H                      (FP64 one-sided Jacobi on the l x l factor)
//   D ~ Q B = (Q Wr) S (Qb Ur)^H        (left vectors Q Wr, right vectors Qb Ur)
//
// The four products with D (m x n) and the two that form the kept singular vectors run on the
// tensor cores with six exact BF16 slices (tc_zgemm.cu); the QR factorisations are the whole-GPU
// Householder kernel (hqr_grid.cu), the l x l SVD the whole-GPU Jacobi (jacobi_grid.cu). The part
// of D outside span(Q) enters the truncation as one lumped singular value ||D - Q Q^H D||_F,
// formed explicitly (D - Q Z^H on the tensor cores, then its Frobenius norm: no cancellation), so
// the discarded weight still counts everything that is dropped.
//
// Every bond's items are written on the device from its live dims (plan kernels), so a CUDA graph
// of the step replays unchanged as the bond dimensions grow.
#include "kernels.h"

namespace ptk {

namespace {

__device__ __forceinline__ void live_shape(const BondWork& W, int* Ma, int* Na) {
  const int mD = W.info[0], nD = W.info[1];
  const bool tr = W.info[2] != 0;
  *Ma = (mD > 0 && nD > 0) ? (tr ? nD : mD) : 0;
  *Na = (mD > 0 && nD > 0) ? (tr ? mD : nD) : 0;
}

__device__ __forceinline__ ZGemmItem zitem(const BondWork& W, const double2* A, int lda, int opA, const double2* B,
                                           int ldb, int opB, double2* C, int ldc, int M, int N, int K,
                                           const int* bcol) {
  ZGemmItem it{};
  it.A = A;
  it.B = B;
  it.C = C;
  it.lda = lda;
  it.ldb = ldb;
  it.ldc = ldc;
  it.M = M;
  it.N = N;
  it.K = K;
  it.opA = opA;
  it.opB = opB;
  it.bcol = bcol;
  it.TA = W.ZA;
  it.TB = W.ZB;
  it.cap_m = W.rs_mx;
  it.cap_n = W.L_cap;
  it.cap_k = W.rs_mx;
  it.flag = nullptr;
  it.acc = 0;
  return it;
}

}  // namespace

// Omega (rows x cols, column-major, ld rows): real and imaginary parts uniform in (-1, 1)
__global__ void k_rsvd_omega(double2* Om, int rows, int cols, unsigned seed) {
  const size_t tot = (size_t)rows * cols;
  const unsigned long long base = (unsigned long long)seed << 40;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x)
    Om[i] = make_double2(hash_unit(base + 2 * i), hash_unit(base + 2 * i + 1));
}

// The range finder's items of every bond (one thread per bond): l = min(n, chi_max + p) into info[9].
__global__ void k_rsvd_plan(const BondWork* work, int n_work, int chi_max, int p, const double2* Om, int ld_om,
                            ZGemmItem* gy1, ZGemmItem* gz1, ZGemmItem* gy2, ZGemmItem* gz2, ZGemmItem* gres,
                            QRItem* q1, QRItem* qz, QRItem* q2, QRItem* qb, int* status) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  live_shape(W, &Ma, &Na);
  int l = (Ma > 0 && Na > 0) ? min(Na, chi_max + p) : 0;
  if (l > W.L_cap || Na > ld_om || Ma > W.rs_mx) {
    // beyond the fast path's buffers: the bond is skipped (it keeps its tensors) and reported
    atomicOr(status, ST_CAPACITY);
    W.info[0] = W.info[1] = 0;
    l = 0;
  }
  if (l == 0) Ma = Na = 0;
  W.info[9] = l;
  W.info[8] = l;        // the rank the SVD works at (the bond log's field)
  gy1[w] = zitem(W, W.A, Ma, ZOP_N, Om, ld_om, ZOP_N, W.RY, max(Ma, 1), Ma, l, Na, nullptr);
  gz1[w] = zitem(W, W.A, Ma, ZOP_C, W.RY, max(Ma, 1), ZOP_N, W.RZ, max(Na, 1), Na, l, Ma, nullptr);
  gy2[w] = zitem(W, W.A, Ma, ZOP_N, W.RZ, max(Na, 1), ZOP_N, W.RY, max(Ma, 1), Ma, l, Na, nullptr);
  // D is packed once into ZA (by the first product, Y = D Omega) and D^H once into ZA2 (a pack-only
  // launch before the power iterations): the later products with D skip their A packing
  gy2[w].skip_a = 1;
  gz1[w].TA = W.ZA2;
  gz1[w].skip_a = 1;
  gz2[w] = gz1[w];
  // D <- D - Q Z^H (Z = D^H Q): what lies outside span(Q), whose norm is the lumped tail
  ZGemmItem r = zitem(W, W.RY, max(Ma, 1), ZOP_N, W.RZ, max(Na, 1), ZOP_C, W.A, max(Ma, 1), Ma, Na, l, nullptr);
  r.cap_n = W.rs_mx;
  r.cap_k = W.L_cap;
  r.acc = -1;
  gres[w] = r;
  q1[w] = QRItem{W.RY, W.RH, W.RR, W.Rtau, Ma, l};
  qz[w] = QRItem{W.RZ, W.RH, W.RR, W.Rtau, Na, l};
  q2[w] = q1[w];
  qb[w] = QRItem{W.RZ, W.RH, W.G64, W.Rtau, Na, l};      // R of Z = D^H Q: the l x l factor
}

// ||A||_F^2 of every bond's A (after the residual step: ||D - Q Q^H D||_F^2) into info[12..13]
// (a double), in two passes with a fixed summation order (the result is reproducible bit for bit):
// block p of bond w sums the p-th of RSVD_FRO_PARTS contiguous chunks of A into part[w][p], then
// one block per bond adds the parts.
__global__ void k_rsvd_fro_part(const BondWork* work, int n_work, double* part) {
  const int w = blockIdx.y, p = blockIdx.x;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  live_shape(W, &Ma, &Na);
  const size_t tot = (size_t)Ma * Na;
  const size_t chunk = (tot + RSVD_FRO_PARTS - 1) / RSVD_FRO_PARTS;
  const size_t lo = min(tot, (size_t)p * chunk), hi = min(tot, lo + chunk);
  double s = 0.0;
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double2 v = W.A[i];
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)w * RSVD_FRO_PARTS + p] = red[0];
}

__global__ void k_rsvd_fro_sum(const BondWork* work, int n_work, const double* part) {
  const int w = blockIdx.x;
  if (w >= n_work) return;
  __shared__ double red[RSVD_FRO_PARTS];
  red[threadIdx.x] = part[(size_t)w * RSVD_FRO_PARTS + threadIdx.x];
  __syncthreads();
  for (int o = RSVD_FRO_PARTS / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *(double*)(work[w].info + 12) = red[0];
}

// After the truncation: the kept left vectors U_D[:, c] = Q Wr[:, perm[c]] (into A) and right
// vectors V_D[:, c] = Qb Ur[:, perm[c]] (into V), c < chi.
__global__ void k_rsvd_plan_vectors(Tables T, const BondWork* work, int n_work, ZGemmItem* gu, ZGemmItem* gv) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  live_shape(W, &Ma, &Na);
  const int l = W.info[9];
  const int chi = (Ma > 0 && l > 0) ? min(T.lam_chi[W.lam_l + 1], l) : 0;
  gu[w] = zitem(W, W.RY, max(Ma, 1), ZOP_N, W.V, max(l, 1), ZOP_N, W.A, max(Ma, 1), chi ? Ma : 0, chi, l, W.perm);
  gv[w] = zitem(W, W.RZ, max(Na, 1), ZOP_N, W.G64, max(l, 1), ZOP_N, W.V, max(Na, 1), chi ? Na : 0, chi, l, W.perm);
}

// the kept vectors now sit in order: perm = identity on the kept columns (the recovery reads
// column perm[c])
__global__ void k_rsvd_perm_reset(Tables T, const BondWork* work, int n_work) {
  const int w = blockIdx.x;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  if (W.info[0] <= 0 || W.info[1] <= 0 || W.info[9] <= 0) return;
  const int chi = T.lam_chi[W.lam_l + 1];
  for (int c = threadIdx.x; c < chi; c += blockDim.x) W.perm[c] = c;
}

void launch_rsvd_omega(double2* Om, int rows, int cols, unsigned seed, cudaStream_t st) {
  k_rsvd_omega<<<4 * 152, 256, 0, st>>>(Om, rows, cols, seed);
}

void launch_rsvd_plan(const Tables& T, const BondWork* work, int n_work, const RsvdLists& L, int chi_max, int p,
                      const double2* Om, int ld_om, cudaStream_t st) {
  k_rsvd_plan<<<(n_work + 127) / 128, 128, 0, st>>>(work, n_work, chi_max, p, Om, ld_om, L.gy1, L.gz1, L.gy2, L.gz2,
                                                     L.gres, L.q1, L.qz, L.q2, L.qb, T.status);
}

void launch_rsvd_tail_norm(const BondWork* work, int n_work, double* part, cudaStream_t st) {
  k_rsvd_fro_part<<<dim3(RSVD_FRO_PARTS, n_work), 256, 0, st>>>(work, n_work, part);
  k_rsvd_fro_sum<<<n_work, RSVD_FRO_PARTS, 0, st>>>(work, n_work, part);
}

void launch_rsvd_vectors(const Tables& T, const BondWork* work, int n_work, const RsvdLists& L, cudaStream_t st) {
  k_rsvd_plan_vectors<<<(n_work + 127) / 128, 128, 0, st>>>(T, work, n_work, L.gu, L.gv);
  launch_zgemm(L.gu, n_work, L.tile_cap, L.m_cap, L.l_cap, T.status, st);
  launch_zgemm(L.gv, n_work, L.tile_cap, L.m_cap, L.l_cap, T.status, st);
  k_rsvd_perm_reset<<<n_work, 128, 0, st>>>(T, work, n_work);
}

}  // namespace ptk
