// Mixed-precision pieces of the fast path's SVD (App. A.2 (f-g)): the bulk Jacobi sweeps run in
// FP32 (58x the FP64 arithmetic rate on GB300); their right factor V32 is re-orthonormalised in
// FP64 by two Newton-Schulz steps X <- X (3I - X^H X) / 2, the matrix is rotated once in FP64,
// A <- D X, and FP64 Jacobi sweeps finish from there (few sweeps: A X is already nearly
// orthogonal). Batched over the bonds of a layer with each bond's live dims read from its info.
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
__device__ void gemm_tile(const double2* A, int lda, bool conjA, const double2* B, int ldb, double2* C, int ldc,
                          int m, int n, int k, int tm, int tn) {
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
      Bs[kk][mm] = (bc < n && br < k) ? B[br + (size_t)bc * ldb] : make_double2(0.0, 0.0);
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

// D (FP64, in A) -> FP32 copy for the bulk sweeps
__global__ void k_mix_to_f32(const BondWork* work, int n_work) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  shape(W, &Ma, &Na);
  const size_t tot = (size_t)Ma * Na;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
    const double2 x = W.A[i];
    W.A32[i] = make_float2((float)x.x, (float)x.y);
  }
}

// V32 -> V (FP64)
__global__ void k_mix_v_to_f64(const BondWork* work, int n_work) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  shape(W, &Ma, &Na);
  const size_t tot = (size_t)Na * Na;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
    const float2 x = W.V32[i];
    W.V[i] = make_double2(x.x, x.y);
  }
}

// op 0: G = V^H V;  op 1: Y = V G;  op 2: Y = A V;  op 3: Y = A V on the first k = info[8]
// columns of V (the pivoted QR's rank)  (grid: tiles x tiles x items)
__global__ void __launch_bounds__(256) k_mix_gemm(const BondWork* work, int n_work, int op) {
  const int w = blockIdx.z;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  shape(W, &Ma, &Na);
  const int tm = blockIdx.x, tn = blockIdx.y;
  const int m = op >= 2 ? Ma : Na, n = op == 3 ? min(W.info[8], Na) : Na;
  if (tm * TB >= m || tn * TB >= n) return;
  if (op == 0) gemm_tile(W.V, Na, true, W.V, Na, W.G64, Na, Na, Na, Na, tm, tn);
  else if (op == 1) gemm_tile(W.V, Na, false, W.G64, Na, W.Y64, Na, Na, Na, Na, tm, tn);
  else gemm_tile(W.A, Ma, false, W.V, Na, W.Y64, Ma, Ma, n, Na, tm, tn);
}

// op 0: V = 1.5 V - 0.5 Y (Newton-Schulz update);  op 1: A = Y (the rotated matrix)
__global__ void k_mix_update(const BondWork* work, int n_work, int op) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  int Ma, Na;
  shape(W, &Ma, &Na);
  const size_t tot = op == 0 ? (size_t)Na * Na : (size_t)Ma * Na;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
    if (op == 0) {
      const double2 v = W.V[i], y = W.Y64[i];
      W.V[i] = make_double2(1.5 * v.x - 0.5 * y.x, 1.5 * v.y - 0.5 * y.y);
    } else {
      W.A[i] = W.Y64[i];
    }
  }
}

// Y64 = A V (A: Ma x Na, V: Na x Na), or only its first info[8] columns (rank_cols)
void launch_mix_gemm_av(const BondWork* work, int n_work, int k_cap, int m_cap, cudaStream_t st, bool rank_cols) {
  const int tk = (k_cap + TB - 1) / TB, tmm = (m_cap + TB - 1) / TB;
  k_mix_gemm<<<dim3(tmm, tk, n_work), 256, 0, st>>>(work, n_work, rank_cols ? 3 : 2);
}

// stage 1: FP32 copy of D and the FP32 bulk sweeps (V32 from identity)
void launch_mixed_fp32(const BondWork* work, int n_work, int blocks, int max_sweeps, unsigned* sync3, int* cnt,
                       int* status, cudaStream_t st) {
  const float eps32 = 5.9604644775390625e-8f;
  k_mix_to_f32<<<dim3(128, n_work), 256, 0, st>>>(work, n_work);
  launch_jacobi_grid(work, n_work, blocks, max_sweeps, sync3, cnt, status, st, /*fp32=*/1, /*init_v=*/1,
                     /*finalize=*/0, eps32, /*sweep_slot=*/6);
}

// stage 2: V <- Newton-Schulz(V32) twice in FP64, then A <- D V
void launch_mixed_reorth(const BondWork* work, int n_work, int k_cap, int m_cap, cudaStream_t st) {
  const int gx = 128;
  k_mix_v_to_f64<<<dim3(gx, n_work), 256, 0, st>>>(work, n_work);
  const int tk = (k_cap + TB - 1) / TB, tmm = (m_cap + TB - 1) / TB;
  for (int it = 0; it < 2; ++it) {
    k_mix_gemm<<<dim3(tk, tk, n_work), 256, 0, st>>>(work, n_work, 0);
    k_mix_gemm<<<dim3(tk, tk, n_work), 256, 0, st>>>(work, n_work, 1);
    k_mix_update<<<dim3(gx, n_work), 256, 0, st>>>(work, n_work, 0);
  }
  k_mix_gemm<<<dim3(tmm, tk, n_work), 256, 0, st>>>(work, n_work, 2);
  k_mix_update<<<dim3(gx, n_work), 256, 0, st>>>(work, n_work, 1);
}

// stage 3: FP64 sweeps from the re-orthonormalised V. Their noise floor reaches below the
// truncation threshold (the caller passes ~1e-2 eps_trunc): the basis of every singular subspace
// the truncation can keep must be the FP64 one, because the trajectory amplifies a change of
// basis there even at singular values of 1e-8 of the largest.
void launch_mixed_fp64(const BondWork* work, int n_work, int blocks, int max_sweeps, unsigned* sync3, int* cnt,
                       int* status, double polish_floor, cudaStream_t st) {
  launch_jacobi_grid(work, n_work, blocks, max_sweeps, sync3, cnt, status, st, /*fp32=*/0, /*init_v=*/0,
                     /*finalize=*/1, polish_floor, /*sweep_slot=*/3);
}

}  // namespace ptk
