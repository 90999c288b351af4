// Kernel declarations shared by the engine and the kernel translation units.
#pragma once
#include "common.cuh"

namespace ptk {

constexpr int QR_THREADS_ = 512;

struct Super4;

__global__ void k_site_contract(Tables T, const SiteWork* work, int n_work);
__global__ void k_site_swap(Tables T, const SiteWork* work, int n_work);
__global__ void k_build_blocks(Tables T, const BondWork* work, int n_work);
__global__ void k_householder(Tables T, const BondWork* work, int n_work);
__global__ void k_theta_gate(Tables T, const BondWork* work, int n_work);
__global__ void k_nan_guard(Tables T, const BondWork* work, int n_work);
constexpr int BOND_LOG_INTS = 10;
__global__ void k_bond_log(Tables T, const BondWork* work, int n_work, int layer, int* log, int cap_steps, int nb);
// the autotuner's synthetic full-capacity state: every Gamma at capacity filled with seeded values
// in (-1, 1), every lambda with a decaying unit-norm profile (dims set by the host beforehand)
__global__ void k_tune_fill(Tables T, int n_sites, int n_lams, unsigned seed);
// rsvd: the singular values are the range finder's l = info[9] values, plus the part of D outside
// its subspace as one lumped value ||D - Q Q^H D||_F (info[12..13]) when l < min(m, n)
__global__ void k_truncate(Tables T, const BondWork* work, int n_work, int chi_max, double eps,
                           double mtol, int rsvd = 0);
__global__ void k_recover(Tables T, const BondWork* work, int n_work);
__global__ void k_caps(Tables T, int n_mpos);
__global__ void k_observe_m(Tables T, int n_chains, double2* Mbuf, const size_t* moff);
__global__ void k_observe(Tables T, int n_chains, const double2* ops, int n_ops, int n_max,
                          double2* obs, double2* trace, double2* Lbuf, double2* Rbuf, int ld,
                          int use_history, const double2* Mbuf, const size_t* moff);
__global__ void k_step_inc(int* step);
__global__ void k_svd_load(const double2* A, int m, int n, int batch, double2* work_A,
                           size_t strideA);
__global__ void k_svd_store(const double2* work_A, const double2* work_V, const double* sig,
                            const int* perm, int m, int n, int batch, size_t strideA,
                            size_t strideV, double* sigma_out, double2* U, double2* V);

// whole-GPU Householder QR/LQ of the outer blocks of every bond of a layer (hqr_grid.cu), and the
// same factorisation over a list of matrices: A (m x n, m >= n, column-major, ld m) is replaced by
// the explicit Q, R (n x n, ld n) receives the triangular factor, H (m x n) and tau (n) are scratch
struct QRItem {
  double2* A;
  double2* H;
  double2* R;
  double* tau;
  int m, n;
};
void launch_hqr_items(const QRItem* items, int n_items, int blocks, unsigned* sync3, int* status, cudaStream_t st);
int hqr_items_ok();
int hqr_grid_ok();
int hqr_grid_fits(int total_cols_cap, int n_items, int blocks);
void launch_hqr_grid(const Tables& T, const BondWork* work, int n_work, int blocks, unsigned* sync3,
                     cudaStream_t st);

// cluster-parallel FP64 bond SVD (jacobi_cluster.cu)
int jacobi_cluster_size(int want);
void launch_jacobi_cluster(const BondWork* work, int n_work, int cluster, int max_sweeps, int* status,
                           cudaStream_t st);

// whole-GPU FP64 bond SVD (jacobi_grid.cu): blocks = one per SM (0 if not co-schedulable);
// sync3: 3 words of device memory (arrival count, unused, abort flag); cnt: 2 ints per item
int jacobi_grid_blocks();
// init_v: start from V = I; finalize: sigma, U, order; floor_eps: unit roundoff of the noise floor;
// sweep_slot: info[] index for the sweep count
// on_b: 1 = B = R^H of the pivoted QR (Na x info[8]), 2 = the range finder's l x l factor in G64
// (l = info[9]); with_v: accumulate V; tol_scale: rotation threshold
// in units of the unit roundoff (0: the row count)
void launch_jacobi_grid(const BondWork* work, int n_work, int blocks, int max_sweeps, unsigned* sync3,
                        int* cnt, int* status, cudaStream_t st, int init_v = 1, int finalize = 1,
                        double floor_eps = 1.1102230246251565e-16, int sweep_slot = 3, int on_b = 0,
                        int with_v = 1, double tol_scale = 0.0);

// QR preconditioning of the bond SVD (qrcp.cu): pivoted QR of D into Y64, B = R^H into G64;
// after the Jacobi on B: V_D = P U', U_D = D V_D / sigma
int qrcp_cluster_size(int want, int m_cap, int n_cap);
int qrcp_smem_cluster(int m_cap, int n_cap);
// whole-GPU variant (cooperative, one CTA per SM): usable when qrcp_grid_ok() and the layer fits
int qrcp_grid_ok();
int qrcp_grid_fits(int n_work, int m_cap, int total_cols_cap, int blocks);
// tau2: squared relative noise level of D at which the pivoted QR stops (rank-revealing);
// kmax: stop after at most kmax reflectors (the autotuner times a prefix; otherwise INT_MAX)
void launch_qrcp_grid(const BondWork* work, int n_work, int blocks, unsigned* sync3, double tau2, int kmax,
                      int* status, cudaStream_t st);
void launch_qrcp_precondition(const BondWork* work, int n_work, int cluster, int smem_cluster, int k_cap, int m_cap,
                              double tau2, int kmax, int* status, cudaStream_t st);
// after the truncation: V_D and U_D on the kept columns (lam_chi: the tables' bond dims)
void launch_qrcp_finish(const BondWork* work, int n_work, int k_cap, int m_cap, const int* lam_chi,
                        cudaStream_t st);
void launch_mix_gemm_av(const BondWork* work, int n_work, int k_cap, int m_cap, const int* lam_chi, cudaStream_t st);

// tensor-core theta + gate of the fast path (tc_theta.cu); precision: 1 TF32x3, 2 BF16x3, 3 TF32x1,
// 4 BF16 fixed-point slices. Packed operand bytes of a bond (which: 0 = A, 1 = B'), its output tile
// capacity, and the launch (pack kernels + the persistent GEMM) over one layer.
size_t tc_pack_bytes(const BondWork& W, int which, int precision);
int tc_tile_cap(const BondWork& W, int precision);
void launch_tc_theta(const Tables& T, const BondWork* work, int n_work, int tile_cap, int precision,
                     cudaStream_t st);

// batched complex GEMM on the tensor cores with an FP64-class result (tc_zgemm.cu):
// C = opA(A) opB(B), M x N, inner dimension K, per item; live dims in device memory (M, N or K = 0:
// the item is skipped and C left untouched). TA / TB: the item's packed operands, sized by
// zgemm_pack_bytes for its capacities (cap_m x cap_k for A, cap_n x cap_k for B).
enum : int { ZOP_N = 0, ZOP_T = 1, ZOP_C = 2 };
struct ZGemmItem {
  const double2* A;
  const double2* B;
  double2* C;
  int lda, ldb, ldc;
  int M, N, K;
  int opA, opB;            // ZOP_N as stored (column-major), ZOP_T transposed, ZOP_C conjugate transpose
  const int* bcol;         // column n of opB(B) is its stored column bcol[n] (NULL: n)
  unsigned char* TA;
  unsigned char* TB;
  int cap_m, cap_n, cap_k;
  int* flag;               // set to 1 when a product entry is not finite (NULL: not reported)
  int acc;                 // 0: C = opA(A) opB(B); -1: C = C - opA(A) opB(B)
  int skip_a;              // 1: A's slice planes and row exponents are already in TA (packed earlier)
};
size_t zgemm_pack_bytes(int rows_cap, int k_cap, int which);
// the A operands' slice planes and row exponents alone (for items whose later products skip them)
void launch_zgemm_pack_a(const ZGemmItem* items, int n_items, int m_cap_max, int* status, cudaStream_t st);
int zgemm_tile_cap(int m_cap, int n_cap);
// tile_cap: total output tiles of the item list at capacity (the persistent grid's upper bound);
// m_cap_max / n_cap_max: the largest M and N capacities (pack grid sizes)
void launch_zgemm(const ZGemmItem* items, int n_items, int tile_cap, int m_cap_max, int n_cap_max, int* status,
                  cudaStream_t st);
// the most items one launch_zgemm takes
int zgemm_max_items();

// the fast path's PT site contraction on the tensor cores (tc_contract.cu): items[w] is site w's GEMM
// (output scratch C, packed planes TA / TB and their capacities set at init; a plan kernel writes the
// operands and live dims every step, so the launch sequence is graph-safe); writes Gamma' into the
// sites' second buffers, to be swapped in by k_site_swap
void launch_site_tc(const Tables& T, const SiteWork* work, int n_work, ZGemmItem* items, int gx, int tile_cap,
                    int m_cap_max, int n_cap_max, cudaStream_t st);
// the fast path's Gamma recovery on the tensor cores (tc_contract.cu): items[2w], items[2w + 1] are
// bond w's left and right products (C in the bond's Householder scratch HH and HH + mL_cap nL_cap,
// packed planes and caps set at init), bcols[w] its column maps (nL_cap + mR_cap ints)
void launch_recover_tc(const Tables& T, const BondWork* work, int n_work, ZGemmItem* items, int* const* bcols,
                       int gx, int tile_cap, int m_cap_max, int n_cap_max, cudaStream_t st);

// the fast path's randomized truncated SVD of every bond of a layer (rsvd.cu): device item lists
// (one entry per bond each) and their launch capacities
struct RsvdLists {
  ZGemmItem *gy1, *gz1, *gy2, *gz2, *gres, *gu, *gv;
  QRItem *q1, *qz, *q2, *qb;
  double* fro_part;        // RSVD_FRO_PARTS doubles per bond: partial sums of the tail norm
  int tile_cap;            // output tiles of one product over the layer at capacity
  int m_cap, l_cap;        // largest row count and range-finder width of the layer's bonds
};
constexpr int RSVD_OVERSAMPLE = 32;
// power iterations: the subspace error at the cut chi falls like (s_{l+1} / s_chi)^(2q+1)
constexpr int RSVD_POWER = 2;
void launch_rsvd_omega(double2* Om, int rows, int cols, unsigned seed, cudaStream_t st);
// the order of a layer: plan (item lists, l into info[9]); gy1 -> QR q1; RSVD_POWER times
// (gz1 -> QR qz, gy2 -> QR q2); gz2; gres (D - Q Z^H); tail norm; QR qb (l x l factor into G64);
// Jacobi on it (launch_jacobi_grid, on_b = 2); truncation (k_truncate, rsvd = 1); vectors
void launch_rsvd_plan(const Tables& T, const BondWork* work, int n_work, const RsvdLists& L, int chi_max, int p,
                      const double2* Om, int ld_om, cudaStream_t st);
// part: RSVD_FRO_PARTS doubles per bond (scratch of the two-pass, fixed-order sum)
constexpr int RSVD_FRO_PARTS = 64;
void launch_rsvd_tail_norm(const BondWork* work, int n_work, double* part, cudaStream_t st);
void launch_rsvd_vectors(const Tables& T, const BondWork* work, int n_work, const RsvdLists& L, cudaStream_t st);

// set the message returned by pt_tebd_last_error(NULL) (engine.cu)
void set_global_error(const char* msg);

// local super-operator launch (struct passed by value lives in the kernel TU)
void launch_apply_local(const Tables& T, int site, int lam, const double2* s16, cudaStream_t st);

}  // namespace ptk
