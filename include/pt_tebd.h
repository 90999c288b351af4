/*
 * pt_tebd.h -- C ABI of the GB300 PT-TEBD time step.
 *
 * PT-TEBD (arXiv:2201.05529) evolves chains of open quantum systems in Liouville space: an
 * augmented MPS in Vidal form, Gamma_n[chi_{n-1}][d^2][kappa_n][chi_n] and lambda_n[chi_n]
 * (App. A.1), is advanced per time step by the second-order splitting of Eq. (propagator-env):
 * a chain half step, the PT-MPO site contractions (App. A.2), and another chain half step,
 * each chain half being O(dt/4) E(dt/2) O(dt/4) layers of two-site Liouville gates applied by
 * the contraction/decomposition sequence of App. A.2 with exact QR reductions and an FP64
 * one-sided Jacobi SVD truncated by the relative rule of App. A.2. Observables are read out by
 * closing the augmented legs with cap tensors (App. A.3) and the Liouville legs with trace or
 * observable vectors; two-time correlations insert a left/right super-operator (App. A.4).
 *
 * Conventions: spin-1/2, d^2 = 4; basis index 0 = up; row-major vectorisation
 * vec(rho)[i*2 + j] = rho[i][j]; Tr(O rho) = vec(O^T) . vec(rho). Complex numbers are stored
 * interleaved (re, im) as doubles. Two-site gates are 16x16 row-major with per-site grouping
 * [(p'_n*4 + p'_{n+1})][(p_n*4 + p_{n+1})].
 *
 * Ownership: every pointer an entry point takes is caller-owned host memory that is copied before
 * the call returns, except `cuda_stream` (borrowed for the handle's lifetime). The library owns
 * all device memory of a handle; it comes from the allocator registered with
 * pt_tebd_set_allocator (e.g. PyTorch's caching allocator), else from cudaMalloc.
 *
 * Errors: every int-returning call returns 0 on success or a negative PT_ERR_* code; the message
 * of the last failure is available from pt_tebd_last_error(). Device-side failures (capacity
 * overflow, SVD non-convergence, NaN) are recorded in a device status word that is read back at
 * every synchronising call (pt_tebd_observe, pt_tebd_read_history, pt_tebd_sync).
 */
#ifndef PT_TEBD_H
#define PT_TEBD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PT_OK 0
#define PT_ERR_ARG (-1)
#define PT_ERR_OOM (-2)
#define PT_ERR_CAPACITY (-3)
#define PT_ERR_SVD_NOCONV (-4)
#define PT_ERR_DEVICE_TIMEOUT (-5)
#define PT_ERR_NAN (-6)
#define PT_ERR_CUDA (-7)
#define PT_ERR_STEPS (-8)

typedef struct pt_tebd* pt_tebd_t;

typedef enum {
  PT_FP64 = 0,      /* every stage in FP64 */
  PT_TF32X3 = 1,    /* theta and the gate as one tensor-core GEMM (the gate folded into the right
                       operand in FP64): each FP64 operand split into three TF32 pieces, the six
                       piece products of order <= 2 accumulated in FP32 (limited by that
                       accumulation to ~1e-6 relative); FP64 SVD, truncation and readout */
  PT_BF16X3 = 2,    /* the same with three BF16 pieces (~24 significant bits) */
  PT_TF32X1 = 3,    /* one TF32 piece, one product (speed reference only) */
  PT_BF16_OZAKI = 4 /* the fast path: every large product on the tensor cores from fixed-point BF16
                       slices (each operand row / column scaled by a power of two and cut into six
                       7-bit slices; the leading slice products sum exactly in FP32 accumulators over
                       K chunks of 512, Ozaki's error-free splitting; ~1e-12 of the operands' scale).
                       theta + gate is one such GEMM; the bond SVD is a randomized truncated SVD
                       (range finder of width l = min(n, chi_max + 32) with two power iterations, its
                       products on the tensor cores, FP64 Householder QR and an FP64 Jacobi SVD of
                       the l x l factor; the part of D outside the range counts as one discarded
                       singular value). Its singular values are accurate to ~1e-11 of sigma_max, so
                       the multiplet rule uses max(multiplet_tol, 1e-9). Truncation, Gamma recovery
                       and readout in FP64 */
} pt_precision;

/* One chain (App. A.1). Sites without a bath have ptmpo_id = -1 (augmented leg of dimension 1).
 * rho0 gives a product initial state; alternatively gamma0/lambda0 give a full augmented MPS
 * (correlated initial chain-environment state, App. A.1): then rho0 may be NULL. */
typedef struct {
  int N;                          /* number of sites, >= 1 */
  const double* rho0;             /* [N][4] complex: vec(rho_n); ignored if gamma0 != NULL */
  const double* gates_q;          /* [N-1][16][16] complex: exp(L^{K'}_b dt/4) */
  const double* gates_h;          /* [N-1][16][16] complex: exp(L^{K'}_b dt/2) */
  const double* local_prop;       /* [N][4][4] complex on-site propagator applied after the PT
                                     tensor at each step, or NULL for none */
  const int* ptmpo_id;            /* [N]: index into pt_mpos, or -1 */
  const int* chi0;                /* [N+1] initial bond dims (chi0[0] = chi0[N] = 1) or NULL */
  const int* kappa0;              /* [N] initial augmented dims or NULL */
  const double* const* gamma0;    /* [N] pointers to Gamma_n[chi0[n]][4][kappa0[n]][chi0[n+1]] complex */
  const double* const* lambda0;   /* [N+1] pointers to real lambda_n[chi0[n]] */
  const double* lognorm0;         /* with gamma0: [N+1] log-norms carried by the bonds (the state is
                                     exp(their sum) times the network; a checkpoint's
                                     pt_tebd_get_lognorms), or NULL for none */
} pt_chain_desc;

/* One PT-MPO (App. A.1; shared by every site whose bath is identical). */
typedef struct {
  int K;                          /* number of time steps it covers */
  const int* kappa;               /* [K+1] bond dims; kappa[0] must match the site's initial kappa */
  const double* const* P;         /* [K] pointers: P^(k+1)[kappa[k]][4][4][kappa[k+1]] complex,
                                     index [a][p_in][p_out][b] */
} pt_mpo_desc;

typedef struct {
  int chi_max;                    /* bond dimension cap */
  double eps;                     /* relative singular value threshold (App. A.2) */
  double multiplet_tol;           /* relative gap below which a cut may not split a multiplet */
  pt_precision precision;
  int max_steps;                  /* history capacity when no PT-MPO bounds the run (0: 1024) */
  int max_sweeps;                 /* Jacobi sweep cap before PT_ERR_SVD_NOCONV (0: 60) */
  int use_graph;                  /* capture one step as a CUDA graph and replay it */
  int autotune;                   /* 1: per bond layer, time the candidate kernels of the SVD's pivoted
                                     QR and of the outer-block QR once, on a synthetic state at
                                     capacity, and keep the fastest (0: a fixed default order) */
  const char* tune_cache;         /* text file of tuned choices (read, appended), or NULL */
  int force_route;                /* 0: tuned or default; else 1 + qr + 4 k2 for every layer, with qr
                                     0 whole-GPU / 1 cluster shared-memory / 2 cluster global-memory
                                     pivoted QR, k2 0 whole-GPU / 1 one-CTA-per-block outer QR
                                     (PT_ERR_ARG where it does not fit) */
} pt_options;

/* Device memory hook: alloc(bytes, ctx) returns device memory or NULL; free(ptr, ctx). */
typedef void* (*pt_alloc_fn)(size_t bytes, void* ctx);
typedef void (*pt_free_fn)(void* ptr, void* ctx);
void pt_tebd_set_allocator(pt_alloc_fn alloc, pt_free_fn free_fn, void* ctx);

/* Build a handle: copies the chains, gates and PT-MPOs to the device, builds the caps (App. A.3)
 * on the device, and prepares the step. cuda_stream is a cudaStream_t (NULL: default stream).
 * Errors: PT_ERR_ARG (malformed descriptors), PT_ERR_CAPACITY (an initial augmented MPS with a bond
 * above chi_max, or a bond block beyond the kernels' limits), PT_ERR_OOM (the allocator returned
 * NULL; everything allocated so far is released), PT_ERR_CUDA. */
int pt_tebd_init(pt_tebd_t* out, const pt_chain_desc* chains, int n_chains,
                 const pt_mpo_desc* pt_mpos, int n_mpos, const pt_options* opt, void* cuda_stream);

/* Register the single-site operators (row-major 2x2 complex, [n_ops][2][2]) whose expectation
 * values Tr(O_n rho) are recorded on every site after every step (and now, at the current step). */
int pt_tebd_set_observables(pt_tebd_t h, const double* ops, int n_ops);

/* Advance every chain by n_steps full steps (asynchronous on the handle's stream). */
int pt_tebd_step(pt_tebd_t h, int n_steps);

/* Expectation values of ops at the current step, synchronously.
 * out: [n_chains][N_max][n_ops] complex (host), raw Tr(O rho) or divided by Tr(rho) if normalize;
 * trace_out: [n_chains] complex (host) or NULL. */
int pt_tebd_observe(pt_tebd_t h, const double* ops, int n_ops, double* out, double* trace_out,
                    int normalize);

/* Recorded values of the registered ops for steps [first, first+count):
 * out [count][n_chains][N_max][n_ops] complex, trace_out [count][n_chains] complex (either NULL). */
int pt_tebd_read_history(pt_tebd_t h, int first, int count, double* out, double* trace_out);

/* Insert rho -> A rho (side 0) or rho -> rho A (side 1) on one site (App. A.4). */
int pt_tebd_apply_local(pt_tebd_t h, int chain, int site, const double* op2x2, int side);

/* State queries (synchronous): number of completed steps; bond dims [N+1] and augmented dims [N]
 * of one chain; lambda of one bond (up to cap doubles); log of the state's norm factor. */
int pt_tebd_steps_done(pt_tebd_t h);
/* Kernel launches of one step: the kernel nodes of the captured step graph (use_graph only). */
int pt_tebd_step_kernels(pt_tebd_t h);
/* The kernels each layer runs (the paper has no counterpart): out8 = [odd qr, odd k2, odd tuned,
 * odd from cache, even qr, even k2, even tuned, even from cache] (routes as in pt_options);
 * ms10 (may be NULL) = the tuner's timings per layer: 3 pivoted-QR and 2 outer-QR candidates (ms,
 * -1 where not a candidate). */
int pt_tebd_get_routes(pt_tebd_t h, int* out8, float* ms10);
/* The tuner's cache file (the paper has no counterpart): one line per layer shape,
 * "key<TAB>qr<TAB>k2<TAB>timings"; the last valid line of a key wins, malformed lines are ignored.
 * lookup returns 1 and the choice if the key is present, 0 if not; store appends a line. No GPU
 * needed. */
int pt_tune_cache_lookup(const char* path, const char* key, int* qr, int* k2);
int pt_tune_cache_store(const char* path, const char* key, int qr, int k2);
/* State of one chain (App. A.1's augmented MPS), synchronous, host outputs owned by the caller; each
 * call also reports a pending device status error. get_dims: chi[0..N] bond dimensions and
 * kappa[0..N-1] augmented dimensions (either may be NULL). get_lambda: the weights of bond `bond`
 * (0..N) into out[0 .. min(chi, cap)), returns chi. get_lognorm: *out = the log-norm the chain has
 * accumulated (the state is exp(*out) times the network); get_lognorms: the same bond by bond,
 * out[0..N] (their sum is get_lognorm's value). PT_ERR_ARG for a bad chain, bond or NULL out. */
int pt_tebd_get_dims(pt_tebd_t h, int chain, int* chi, int* kappa);
int pt_tebd_get_lambda(pt_tebd_t h, int chain, int bond, double* out, int cap);
int pt_tebd_get_lognorm(pt_tebd_t h, int chain, double* out);
int pt_tebd_get_lognorms(pt_tebd_t h, int chain, double* out);

/* Checkpoint read of one site tensor (App. B.2 continues a propagation from the full augmented MPS):
 * copies Gamma_n of `site` (0-based) of `chain` into out as complex [chi_{n-1}][4][kappa_n][chi_n]
 * (interleaved re, im; the live dims of pt_tebd_get_dims), the layout pt_chain_desc.gamma0 takes.
 * cap is out's size in complex elements; out may be NULL to ask for the size. Synchronous; returns
 * the element count, PT_ERR_ARG when cap is too small. Together with pt_tebd_get_lambda and
 * pt_tebd_get_lognorms it gives a resumable state: a new handle initialised with these tensors as
 * gamma0 / lambda0, the log-norms as lognorm0, and every PT-MPO cut at the current step (its tensors
 * from P^(k+1) on, kappa[0] = the site's current kappa) continues the same run: bit for bit when the
 * cut PT-MPOs keep their largest bond (the new handle then has the same capacities, kernel routes and
 * sketch matrix). */
int pt_tebd_get_gamma(pt_tebd_t h, int chain, int site, double* out, size_t cap);

/* Jacobi sweeps of the most recent update of every bond (odd-layer bonds first, then even):
 * out[2i] = FP64 sweeps (negative: the bond hit max_sweeps), out[2i+1] = the update's fault flags
 * (1: theta + gate gave a NaN or an infinity, 2: a NaN singular value, 4: the kept singular values
 * have norm zero; 0 normally). Writes min(cap, n_bonds) pairs; returns n_bonds. */
int pt_tebd_get_svd_sweeps(pt_tebd_t h, int* out, int cap);

/* Per-step log of every bond update (the bond dimensions over time that App. B.3 tracks, plus the
 * SVD's work), for steps [first, first+count): out receives [count][6 layers][nb][10] ints, layers in
 * step order O E O | O E O (O: bonds (1,2),(3,4),..., E: the others), bond b of the layer's list
 * (chains in order, bonds left to right); nb = the larger list length, absent bonds all zero. Fields:
 * 0 rows and 1 columns of D (0: skipped), 2 the pivoted QR's rank (0 on routes without it),
 * 3 Jacobi sweeps (negative: the sweep cap was hit), 4 fault flags (as in pt_tebd_get_svd_sweeps),
 * 5 the new bond dimension, 6 and 7 the augmented dimensions of the two sites, 8-9 the discarded
 * weight ||sigma_discarded||_2 / sigma_max as a double. cap_ints bounds out. Synchronous; returns
 * nb. A diagnostic: it also reads after a device status error (PT_ERR_NAN and the like), whose
 * bond it shows; only a CUDA error fails it. */
int pt_tebd_read_bond_log(pt_tebd_t h, int first, int count, int* out, size_t cap_ints);

/* Copy the whole device state into a new handle (App. B.2: continue from the full augmented MPS). */
int pt_tebd_clone(pt_tebd_t h, pt_tebd_t* out);

/* Wait for the stream and check the device status word. */
int pt_tebd_sync(pt_tebd_t h);

int pt_tebd_destroy(pt_tebd_t h);
const char* pt_tebd_last_error(pt_tebd_t h);   /* h may be NULL: last global error */

/* Per-stage device time of the last pt_tebd_step call with timing enabled, in milliseconds:
 * [0] site contraction, [1] block build + outer-block QR, [2] theta + gate, [3] SVD Jacobi sweeps,
 * [4] truncation, [5] Gamma recovery, [6] readout, [7] the fast path's range-finder Householder
 * QRs, [8] FP64 path: pivoted QR and the U = D V / sigma finish; fast path: the tensor-core
 * products of the randomized SVD (sketches, projection, residual, kept vectors). Timing mode
 * launches eagerly (no graph). */
int pt_tebd_set_timing(pt_tebd_t h, int enable);
int pt_tebd_get_timing(pt_tebd_t h, double* ms9);

/* ---- kernel-level entry points (single operations on device buffers, for unit tests) ---- */

/* Batched FP64 SVD (the one-sided Jacobi of the bond update, App. A.2) of `batch` complex
 * matrices A_b [m][n] row-major (device). Writes singular values sigma [batch][min(m,n)]
 * (descending), U [batch][m][min(m,n)] and V [batch][n][min(m,n)] (device, row-major), so
 * A_b = U diag(sigma) V^H. scratch: device workspace of pt_svd_scratch_bytes(m, n, batch) bytes.
 * Returns PT_ERR_SVD_NOCONV if a matrix did not converge within max_sweeps. */
size_t pt_svd_scratch_bytes(int m, int n, int batch);
int pt_svd_f64(const double* A, int m, int n, int batch, double* sigma, double* U, double* V,
               void* scratch, int max_sweeps, void* cuda_stream);

/* Batched FP64 Householder QR with the explicit Q (the whole-GPU kernel of the outer-block
 * reductions, App. A.2, and of the fast path's range finder): A_b (m x n complex,
 * column-major, 1 <= n <= m, b < batch, contiguous) is replaced by Q_b (m x n, orthonormal columns),
 * R_b (n x n, column-major, upper triangular) is written, A_b(in) = Q_b R_b. scratch: device workspace
 * of pt_qr_scratch_bytes(m, n, batch) bytes. Synchronous. Errors: PT_ERR_ARG, PT_ERR_CAPACITY
 * (n x batch above the kernel's column capacity), PT_ERR_DEVICE_TIMEOUT (a bounded barrier wait). */
size_t pt_qr_scratch_bytes(int m, int n, int batch);
int pt_qr_f64(double* A, int m, int n, int batch, double* R, void* scratch, void* cuda_stream);

/* Batched complex GEMM of the fast path on the tensor cores (the products of the fast path's bond
 * SVD, App. A.2): C_b = opA(A_b) opB(B_b), b < batch, C_b m x n, inner dimension k. Every
 * matrix is complex double (interleaved re, im), column-major, with the given leading dimension
 * (in complex elements) and batch stride (in complex elements); op: 0 as stored, 1 transposed,
 * 2 conjugate transposed. Arithmetic: each row of opA(A) and column of opB(B) is scaled by a power
 * of two and cut into six BF16 fixed-point slices; slice products accumulate in FP32 on the
 * tcgen05 tensor cores (exactly for the two leading levels) and are summed in FP64, so C is
 * accurate to ~1e-12 of max|row of opA(A)| x max|column of opB(B)|. scratch: device workspace of
 * pt_zgemm_scratch_bytes(m, n, k, batch) bytes. Synchronous. Errors: PT_ERR_ARG (bad sizes, op or
 * leading dimension, batch > 1024), PT_ERR_DEVICE_TIMEOUT (a bounded pipeline wait expired). */
size_t pt_zgemm_scratch_bytes(int m, int n, int k, int batch);
int pt_zgemm_sliced(int opA, int opB, int m, int n, int k, const double* A, int lda, long long strideA,
                    const double* B, int ldb, long long strideB, double* C, int ldc, long long strideC, int batch,
                    void* scratch, void* cuda_stream);

/* ---- allocation-free variant of pt_svd_f64 (the paper has no counterpart) ----
 * For callers that cannot allocate device memory: their device memory is owned by another pool
 * (a framework that reserves the GPU up front, a fixed-budget service), or a device allocation is
 * not acceptable where they run (cudaMalloc may synchronise the device and can fail mid-job).
 * Same batched FP64 Jacobi SVD and the same arguments and outputs as pt_svd_f64, minus the
 * scratch pointer: the workspace is a static device array of PT_SVD_NOALLOC_MAX_BYTES bytes that
 * every GPU which loads this library holds until the process exits. A problem whose workspace
 * (pt_svd_scratch_bytes(m, n, batch)) is larger is rejected with PT_ERR_CAPACITY. The first call on
 * a device looks up the array's device address with that device current and caches it per device
 * index (a cudaDeviceReset invalidates it). All calls share the one array: calls that overlap on the
 * GPU race and corrupt each other, so the caller must serialise them. Each call clears what must
 * start at zero, reads the status word back and synchronises the stream before returning, so it
 * must not be called while that stream is being captured. Messages: pt_tebd_last_error(NULL). */
#define PT_SVD_NOALLOC_MAX_BYTES ((size_t)16 << 20)
int pt_svd_f64_noalloc(const double* A, int m, int n, int batch, double* sigma, double* U, double* V,
                       int max_sweeps, void* cuda_stream);

/* ---- diagnostic (the paper has no counterpart) ----
 * Exercises the failure path of the bounded grid barrier used by the cooperative kernels (Jacobi
 * rounds, pivoted-QR steps) without a GPU fault: one CTA per SM runs three barriers with a wait limit
 * of limit_ms (0 < limit_ms <= 10000); withheld_block (-1: none) is a CTA that never arrives. With
 * no CTA withheld the call returns PT_OK; with one withheld the others time out, record the
 * timeout, raise the abort flag and return, and the call returns PT_ERR_DEVICE_TIMEOUT; in both
 * cases the context stays usable. device_status (may be NULL) receives the device status bits.
 * Uses static device variables only and synchronises the device. */
int pt_selftest_grid_barrier(int withheld_block, double limit_ms, int* device_status);

#ifdef __cplusplus
}
#endif

#endif /* PT_TEBD_H */
