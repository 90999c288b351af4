// FP64 GEMM of the SVD's finish (App. A.2): U_D = D V_D on the columns the truncation keeps,
// batched over the bonds of a layer with each bond's live dims read from its info words.
#include "kernels.h"

namespace ptk {

namespace {

__device__ __forceinline__ void shape(const BondWork& W, int* Ma, int* Na) {
  const int mD = W.info[0], nD = W.info[1];
  const bool tr = W.info[2] != 0;
  *Ma = (mD > 0 && nD > 0) ? (tr ? nD : mD) : 0;
  *Na = (mD > 0 && nD > 0) ? (tr ? mD : nD) : 0;
}

constexpr int TB = 32;   // GEMM tile
constexpr int TK = 16;   // GEMM K tile

// C[m x n] = op(A)[m x k] * B[k x n], column-major; op = conjugate transpose if conjA.
// 256 threads, each computes a 2 x 2 block of a 32 x 32 tile.
// bcol: column c of B is column bcol[c] of the stored matrix (NULL: c)
__device__ void gemm_tile(const double2* A, int lda, bool conjA, const double2* B, int ldb, double2* C, int ldc,
                          int m, int n, int k, int tm, int tn, const int* bcol = nullptr) {
  __shared__ double2 As[TK][TB + 1];
  __shared__ double2 Bs[TK][TB + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double2 acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < k; k0 += TK) {
    for (int e = threadIdx.x; e < TK * TB; e += blockDim.x) {
      const int kk = e / TB, mm = e % TB;
      const int row = tm * TB + mm, col = k0 + kk;
      double2 a = make_double2(0.0, 0.0);
      if (row < m && col < k) {
        if (conjA) {
          const double2 x = A[col + (size_t)row * lda];     // (A^H)[row, col] = conj(A[col, row])
          a = make_double2(x.x, -x.y);
        } else {
          a = A[row + (size_t)col * lda];
        }
      }
      As[kk][mm] = a;
      const int bc = tn * TB + mm, br = k0 + kk;
      Bs[kk][mm] = (bc < n && br < k) ? B[br + (size_t)(bcol ? bcol[bc] : bc) * ldb] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      double2 a[2], b[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) a[i] = As[kk][ty * 2 + i];
#pragma unroll
      for (int j = 0; j < 2; ++j) b[j] = Bs[kk][tx * 2 + j];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int row = tm * TB + ty * 2 + i, col = tn * TB + tx * 2 + j;
      if (row < m && col < n) C[row + (size_t)col * ldc] = acc[i][j];
    }
}

}  // namespace

// Y64[:, c] = A V[:, perm[c]] for the kept columns c < lam_chi[bond] (grid: tiles x tiles x items)
__global__ void __launch_bounds__(256) k_mix_gemm(const BondWork* work, int n_work, const int* lam_chi) {
  const int w = blockIdx.z;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  shape(W, &Ma, &Na);
  const int tm = blockIdx.x, tn = blockIdx.y;
  const int n = min(lam_chi[W.lam_l + 1], Na);
  if (tm * TB >= Ma || tn * TB >= n) return;
  gemm_tile(W.A, Ma, false, W.V, Na, W.Y64, Ma, Ma, n, Na, tm, tn, W.perm);
}

void launch_mix_gemm_av(const BondWork* work, int n_work, int k_cap, int m_cap, const int* lam_chi, cudaStream_t st) {
  const int tk = (k_cap + TB - 1) / TB, tmm = (m_cap + TB - 1) / TB;
  k_mix_gemm<<<dim3(tmm, tk, n_work), 256, 0, st>>>(work, n_work, lam_chi);
}

}  // namespace ptk
