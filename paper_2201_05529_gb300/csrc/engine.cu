// Host engine and C ABI of the PT-TEBD step (see include/pt_tebd.h).
//
// One handle holds every chain of a batch. Device state lives in capacity-sized buffers whose
// live dimensions (chi per bond, kappa per site) are read by the kernels from device memory, so a
// whole step -- three bond layers, the PT site layer, three bond layers, readout -- is one fixed
// launch sequence that can be captured as a CUDA graph and replayed.
#include <algorithm>
#include <functional>
#include <climits>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"
#include "../../include/pt_tebd.h"

using cplx = std::complex<double>;

namespace {

pt_alloc_fn g_alloc = nullptr;
pt_free_fn g_free = nullptr;
void* g_ctx = nullptr;
thread_local std::string g_err;

// NVTX range over a host scope (a tracing tool, when one is attached, sees the step's stages and the
// kernel launches inside them; without a tool the calls do nothing)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct HostChain {
  int N;
  std::vector<cplx> rho0;                 // N*4
  std::vector<cplx> gq, gh;               // (N-1)*256
  std::vector<cplx> local_prop;           // N*16 or empty
  std::vector<int> mpo;                   // N
  std::vector<int> chi0, kappa0;          // optional
  std::vector<std::vector<cplx>> gamma0;  // optional
  std::vector<std::vector<double>> lambda0;
  std::vector<double> lognorm0;           // optional: initial log-norm of each bond (N+1)
};

struct HostMpo {
  int K;
  std::vector<int> kappa;                 // K+1
  std::vector<std::vector<cplx>> P;       // K tensors
};

struct Alloc {
  void* p;
  size_t bytes;
};

}  // namespace

struct pt_tebd {
  cudaStream_t stream = nullptr;
  pt_options opt{};
  std::string err;
  std::vector<Alloc> allocs;

  // problem copy (for clone)
  std::vector<HostChain> chains;
  std::vector<HostMpo> mpos_in;

  // layout
  int n_chains = 0, n_sites = 0, n_lams = 0, n_max = 0;
  std::vector<int> site0, lam0;
  std::vector<int> lam_cap_h;
  std::vector<size_t> site_cap_h;
  std::vector<int> kcap_h;            // per site
  std::vector<int> kap_init_h, chi_init_h;   // initial augmented and bond dims (restored after tuning)
  std::vector<int> site_mpo_h;        // per site (after fusion)
  int n_mpos = 0;                     // device PT-MPOs (after fusion)
  int K_limit = 0;

  // device tables
  Tables T{};
  std::vector<double2*> gam_a, gam_b;  // host copies of the buffer pointers (primary/secondary)
  std::vector<double*> lam_buf;
  BondWork* d_odd = nullptr;
  BondWork* d_even = nullptr;
  int n_odd = 0, n_even = 0;
  int gx_bond = 1;
  int cl_odd = 1, cl_even = 1;        // Jacobi cluster sizes per layer list
  int grid_blocks = 0;                // whole-GPU Jacobi: CTAs per launch (0: use the cluster kernel)
  int tiles_odd = 1, tiles_even = 1;  // fast path: theta + gate GEMM output tiles per layer (capacity)
  std::vector<int*> bond_info;        // per bond (odd list, then even list): its info words
  int qr_cluster = 1;                 // CTAs per matrix of the global-memory cluster pivoted QR
  int qr_smem_cluster = 0;            // >0: the cluster shared-memory pivoted QR fits (CTAs per matrix)
  bool qr_grid_odd = false, qr_grid_even = false;   // the whole-GPU pivoted QR fits the layer
  bool hqr_odd = false, hqr_even = false;            // the whole-GPU outer-block QR/LQ fits the layer
  // the kernels each layer runs (chosen by the autotuner, forced, or by the default order)
  struct Route {
    int qr = 2;      // pivoted QR of the SVD: 0 whole GPU, 1 cluster shared memory, 2 cluster global memory
    int k2 = 1;      // outer-block QR/LQ: 0 whole GPU, 1 one CTA per block
    float ms_qr[3] = {-1, -1, -1}, ms_k2[2] = {-1, -1};   // tuner timings (ms; -1: not a candidate)
    bool tuned = false, cached = false;
  } route_odd, route_even;
  int tune_status = 0;                // device status word seen at the end of the tuning run
  int kcap_odd = 1, kcap_even = 1, mcap_odd = 1, mcap_even = 1;
  // fast path: the randomized truncated SVD of the bonds (rsvd.cu)
  bool use_rsvd = false;
  ptk::RsvdLists rs_odd{}, rs_even{};
  double2* d_omega = nullptr;         // the range finder's sketch matrix (ld_omega x l_max)
  int ld_omega = 1;
  unsigned* d_sync3 = nullptr;        // grid barrier state
  int* d_cnt_odd = nullptr;           // per-item rotation counters
  int* d_cnt_even = nullptr;
  SiteWork* d_sites = nullptr;
  int n_site_work = 0;
  int gx_site = 1;
  // fast path: the site layer as one sliced tensor-core GEMM, one item per site (tc_contract.cu)
  ptk::ZGemmItem* d_site_items = nullptr;
  int site_tile_cap = 0, site_mcap = 1, site_ncap = 1;
  // fast path: the Gamma recovery as sliced tensor-core GEMMs, two items per bond (tc_contract.cu)
  struct RecList {
    ptk::ZGemmItem* items = nullptr;
    int** bcols = nullptr;
    int tile_cap = 0, mcap = 1, ncap = 1;
  } rec_odd, rec_even;

  // observables
  double2* d_ops = nullptr;
  int n_ops = 0;
  double2* d_hist = nullptr;
  double2* d_hist_tr = nullptr;
  int hist_cap = 0;
  double2* d_ops_now = nullptr;
  double2* d_obs_now = nullptr;
  double2* d_tr_now = nullptr;
  double2* d_Lbuf = nullptr;
  double2* d_Rbuf = nullptr;
  double2* d_Mbuf = nullptr;          // readout: site tensors with the augmented leg closed
  size_t* d_moff = nullptr;           // [n_sites] offsets into d_Mbuf
  int gx_m = 1;
  int ld = 1;
  static constexpr int MAX_OPS = 16;

  int steps_done = 0;
  int* d_blog = nullptr;              // bond log [hist_cap][6][blog_nb][BOND_LOG_INTS]
  int graph_kernels = 0;              // kernel nodes of the captured step graph
  int blog_nb = 1;
  cudaGraphExec_t graph = nullptr;
  bool timing = false;
  double stage_ms[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  size_t ev_used = 0;

  int fail(int code, const std::string& msg) {
    err = msg;
    g_err = msg;
    return code;
  }

  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (g_alloc) {
      p = g_alloc(bytes, g_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      p = nullptr;
    }
    if (p) allocs.push_back({p, bytes});
    return p;
  }

  void release() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    for (auto& e : ev) {
      cudaEventDestroy(e.second.first);
      cudaEventDestroy(e.second.second);
    }
    ev.clear();
    if (stream) cudaStreamSynchronize(stream);
    for (auto& a : allocs) {
      if (g_free) g_free(a.p, g_ctx);
      else cudaFree(a.p);
    }
    allocs.clear();
  }
};

namespace {

template <class T>
T* upload(pt_tebd* h, const T* src, size_t n) {
  T* d = (T*)h->dalloc(sizeof(T) * n);
  if (!d) return nullptr;
  if (n && cudaMemcpyAsync(d, src, sizeof(T) * n, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return nullptr;
  return d;
}

template <class T>
T* upload(pt_tebd* h, const std::vector<T>& v) {
  return upload(h, v.data(), v.size());
}

int check_cuda(pt_tebd* h, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return h->fail(PT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return PT_OK;
}

int read_status(pt_tebd* h) {
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, h->T.status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->fail(PT_ERR_CUDA, std::string("sync: ") + cudaGetErrorString(e));
  if (st & ST_CAPACITY) return h->fail(PT_ERR_CAPACITY, "device: live dimension exceeded a buffer capacity");
  if (st & ST_SVD_NOCONV) return h->fail(PT_ERR_SVD_NOCONV, "device: Jacobi SVD did not converge within max_sweeps");
  if (st & ST_NAN) return h->fail(PT_ERR_NAN, "device: NaN in singular values or norms");
  if (st & ST_PT_RANGE) return h->fail(PT_ERR_STEPS, "device: step beyond the PT-MPO length");
  if (st & ST_TIMEOUT) return h->fail(PT_ERR_DEVICE_TIMEOUT, "device: a grid barrier wait ran out of time");
  return PT_OK;
}

// ---------------------------------------------------------------- timing helpers
void ev_begin(pt_tebd* h, int cat, cudaEvent_t* end_out) {
  if (!h->timing) return;
  if (h->ev_used == h->ev.size()) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    h->ev.push_back({cat, {a, b}});
  }
  auto& e = h->ev[h->ev_used++];
  e.first = cat;
  cudaEventRecord(e.second.first, h->stream);
  *end_out = e.second.second;
}
void ev_end(pt_tebd* h, cudaEvent_t e) {
  if (h->timing) cudaEventRecord(e, h->stream);
}

// ---------------------------------------------------------------- the step launch sequence
// outer-block QR/LQ of a layer: 0 whole GPU (k_hqr_grid), 1 one CTA per block (k_householder)
void enqueue_k2(pt_tebd* h, const BondWork* work, int n, int k2) {
  if (k2 == 0) ptk::launch_hqr_grid(h->T, work, n, h->grid_blocks, h->d_sync3, h->stream);
  else ptk::k_householder<<<dim3(n, 2), ptk::QR_THREADS_, 0, h->stream>>>(h->T, work, n);
}

// pivoted QR of the SVD: 0 whole GPU, 1 cluster shared memory, 2 cluster global memory; it stops at
// D's noise level (FP64 rounding, or the sliced tensor-core product's) or after kmax reflectors
void enqueue_qr(pt_tebd* h, const BondWork* work, int n, int qr, int kmax) {
  const int kc = work == h->d_odd ? h->kcap_odd : h->kcap_even, mc = work == h->d_odd ? h->mcap_odd : h->mcap_even;
  const double tau2 = h->opt.precision == PT_BF16_OZAKI ? 8.271806125530277e-25    // (2^-40)^2
                                                        : 1.232595164407831e-32;   // (2^-53)^2
  if (qr == 0) ptk::launch_qrcp_grid(work, n, h->grid_blocks, h->d_sync3, tau2, kmax, h->T.status, h->stream);
  else
    ptk::launch_qrcp_precondition(work, n, h->qr_cluster, qr == 1 ? h->qr_smem_cluster : 0, kc, mc, tau2, kmax,
                                  h->T.status, h->stream);
}

// multiplet floor of the fast path (relative to sigma_max): above its singular values' accuracy
constexpr double FAST_MULTIPLET_TOL = 1e-9;

void enqueue_layer(pt_tebd* h, const BondWork* work, int n, int layer) {
  if (n == 0) return;
  NvtxRange nv(work == h->d_odd ? "pt_tebd bond layer (odd bonds)" : "pt_tebd bond layer (even bonds)");
  cudaStream_t s = h->stream;
  cudaEvent_t e = nullptr;
  ev_begin(h, 1, &e);
  ptk::k_build_blocks<<<dim3(h->gx_bond, n), 256, 0, s>>>(h->T, work, n);
  const pt_tebd::Route& rt = work == h->d_odd ? h->route_odd : h->route_even;
  enqueue_k2(h, work, n, rt.k2);
  ev_end(h, e);
  ev_begin(h, 2, &e);
  if (h->opt.precision == PT_FP64)
    ptk::k_theta_gate<<<dim3(h->gx_bond, n), 128, 0, s>>>(h->T, work, n);
  else
    ptk::launch_tc_theta(h->T, work, n, work == h->d_odd ? h->tiles_odd : h->tiles_even, (int)h->opt.precision, s);
  ptk::k_nan_guard<<<(n + 127) / 128, 128, 0, s>>>(h->T, work, n);
  ev_end(h, e);
  int* cnt = work == h->d_odd ? h->d_cnt_odd : h->d_cnt_even;
  if (h->use_rsvd) {
    // fast path: randomized truncated SVD (tensor-core products, whole-GPU QR and l x l Jacobi)
    const ptk::RsvdLists& L = work == h->d_odd ? h->rs_odd : h->rs_even;
    const int mc = L.m_cap, lc = L.l_cap;
    int* st = h->T.status;
    // timing categories: 8 the tensor-core products, 7 the Householder QRs of the range finder
    auto gemm = [&](const ptk::ZGemmItem* it, int ncap) {
      ev_begin(h, 8, &e);
      ptk::launch_zgemm(it, n, L.tile_cap, mc, ncap, st, s);
      ev_end(h, e);
    };
    auto qr = [&](const ptk::QRItem* it) {
      ev_begin(h, 7, &e);
      ptk::launch_hqr_items(it, n, h->grid_blocks, h->d_sync3, st, s);
      ev_end(h, e);
    };
    ev_begin(h, 8, &e);
    ptk::launch_rsvd_plan(h->T, work, n, L, h->opt.chi_max, ptk::RSVD_OVERSAMPLE, h->d_omega, h->ld_omega, s);
    ev_end(h, e);
    gemm(L.gy1, lc);                                    // Y = D Omega (packs D)
    ev_begin(h, 8, &e);
    ptk::launch_zgemm_pack_a(L.gz1, n, mc, st, s);      // D^H, packed once for every D^H Q
    ev_end(h, e);
    qr(L.q1);
    for (int it = 0; it < ptk::RSVD_POWER; ++it) {
      gemm(L.gz1, lc);                                  // Z = D^H Q
      qr(L.qz);
      gemm(L.gy2, lc);                                  // Y = D Qz
      qr(L.q2);
    }
    gemm(L.gz2, lc);                                    // Z = D^H Q = B^H
    gemm(L.gres, mc);                                   // D - Q Z^H
    ev_begin(h, 8, &e);
    ptk::launch_rsvd_tail_norm(work, n, L.fro_part, s);
    ev_end(h, e);
    qr(L.qb);                                           // Z = Qb Rb
    ev_begin(h, 3, &e);
    const double tol_scale = 9.007199254740992e6;     // |cos| <= 1e-9, below the products' accuracy
    ptk::launch_jacobi_grid(work, n, h->grid_blocks, h->opt.max_sweeps, h->d_sync3, cnt, h->T.status, s, 1, 1,
                            1.1102230246251565e-16, 3, /*on_b=*/2, /*with_v=*/1, tol_scale);
    ev_end(h, e);
    ev_begin(h, 4, &e);
    // the fast path's singular values carry errors of ~1e-11 of sigma_max: gaps below the
    // FAST_MULTIPLET_TOL floor count as degenerate, so it sees the exact multiplets the FP64 path sees
    const double mtol = std::max(h->opt.multiplet_tol, FAST_MULTIPLET_TOL);
    ptk::k_truncate<<<(n + 63) / 64, 64, 0, s>>>(h->T, work, n, h->opt.chi_max, h->opt.eps, mtol, /*rsvd=*/1);
    ev_end(h, e);
    ev_begin(h, 8, &e);
    ptk::launch_rsvd_vectors(h->T, work, n, L, s);
    ev_end(h, e);
  } else if (h->grid_blocks > 0) {
    // QR-preconditioned FP64 Jacobi: pivoted QR, Jacobi on R^H, then V_D = P U', U_D = D V_D / sigma
    const int kc = work == h->d_odd ? h->kcap_odd : h->kcap_even, mc = work == h->d_odd ? h->mcap_odd : h->mcap_even;
    ev_begin(h, 8, &e);
    enqueue_qr(h, work, n, rt.qr, INT_MAX);
    ev_end(h, e);
    ev_begin(h, 3, &e);
    // rotation threshold |cos(b_i, b_j)| > m u in FP64; the sliced fast path, whose D is accurate to
    // ~1e-12 of its scale, stops its sweeps at |cos| <= 1e-9 (the last, refining sweeps of the
    // quadratic convergence are below its own accuracy)
    const double tol_scale = h->opt.precision == PT_BF16_OZAKI ? 9.007199254740992e6 /* 1e-9 / u */ : 0.0;
    ptk::launch_jacobi_grid(work, n, h->grid_blocks, h->opt.max_sweeps, h->d_sync3, cnt, h->T.status, s, 1, 1,
                            1.1102230246251565e-16, 3, /*on_b=*/1, /*with_v=*/0, tol_scale);
    ev_end(h, e);
  } else {
    // no co-resident whole-GPU launch possible on this device: one thread-block cluster per matrix
    ev_begin(h, 3, &e);
    ptk::launch_jacobi_cluster(work, n, work == h->d_odd ? h->cl_odd : h->cl_even, h->opt.max_sweeps,
                               h->T.status, s);
    ev_end(h, e);
  }
  if (!h->use_rsvd) {
    ev_begin(h, 4, &e);
    ptk::k_truncate<<<(n + 63) / 64, 64, 0, s>>>(h->T, work, n, h->opt.chi_max, h->opt.eps,
                                                  h->opt.multiplet_tol);
    ev_end(h, e);
  }
  if (!h->use_rsvd && h->grid_blocks > 0) {
    // the SVD's finish on the kept columns only: V_D = P U', U_D = D V_D / sigma
    const int kc = work == h->d_odd ? h->kcap_odd : h->kcap_even, mc = work == h->d_odd ? h->mcap_odd : h->mcap_even;
    ev_begin(h, 8, &e);
    ptk::launch_qrcp_finish(work, n, kc, mc, h->T.lam_chi, s);
    ev_end(h, e);
  }
  ev_begin(h, 5, &e);
  const pt_tebd::RecList& RL = work == h->d_odd ? h->rec_odd : h->rec_even;
  if (RL.items)
    ptk::launch_recover_tc(h->T, work, n, RL.items, RL.bcols, h->gx_bond, RL.tile_cap, RL.mcap, RL.ncap, s);
  else
    ptk::k_recover<<<dim3(h->gx_bond, n), 256, 0, s>>>(h->T, work, n);
  ev_end(h, e);
  ptk::k_bond_log<<<(n + 127) / 128, 128, 0, s>>>(h->T, work, n, layer, h->d_blog, h->hist_cap, h->blog_nb);
}

void enqueue_chain_half(pt_tebd* h, int first_layer) {
  enqueue_layer(h, h->d_odd, h->n_odd, first_layer);
  enqueue_layer(h, h->d_even, h->n_even, first_layer + 1);
  enqueue_layer(h, h->d_odd, h->n_odd, first_layer + 2);
}

void enqueue_observe_history(pt_tebd* h) {
  if (h->n_ops == 0) return;
  NvtxRange nv("pt_tebd readout");
  cudaEvent_t e = nullptr;
  ev_begin(h, 6, &e);
  ptk::k_observe_m<<<dim3(h->gx_m, h->n_chains, h->n_max), 256, 0, h->stream>>>(h->T, h->n_chains, h->d_Mbuf,
                                                                                  h->d_moff);
  ptk::k_observe<<<h->n_chains, 256, 0, h->stream>>>(h->T, h->n_chains, h->d_ops, h->n_ops, h->n_max,
                                                     h->d_hist, h->d_hist_tr, h->d_Lbuf, h->d_Rbuf,
                                                     h->ld, 1, h->d_Mbuf, h->d_moff);
  ev_end(h, e);
}

void enqueue_step(pt_tebd* h) {
  enqueue_chain_half(h, 0);
  if (h->n_site_work > 0) {
    NvtxRange nv("pt_tebd site layer");
    cudaEvent_t e = nullptr;
    ev_begin(h, 0, &e);
    if (h->d_site_items)
      ptk::launch_site_tc(h->T, h->d_sites, h->n_site_work, h->d_site_items, h->gx_site, h->site_tile_cap,
                          h->site_mcap, h->site_ncap, h->stream);
    else
      ptk::k_site_contract<<<dim3(h->gx_site, h->n_site_work), 256, 0, h->stream>>>(h->T, h->d_sites,
                                                                                   h->n_site_work);
    ptk::k_site_swap<<<(h->n_site_work + 127) / 128, 128, 0, h->stream>>>(h->T, h->d_sites,
                                                                          h->n_site_work);
    ev_end(h, e);
  }
  enqueue_chain_half(h, 3);
  ptk::k_step_inc<<<1, 1, 0, h->stream>>>(h->T.step);
  enqueue_observe_history(h);
}

int capture_graph(pt_tebd* h) {
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  cudaGraph_t g;
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
    return h->fail(PT_ERR_CUDA, "graph: stream create");
  cudaStream_t keep = h->stream;
  h->stream = cap;
  bool t = h->timing;
  h->timing = false;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_step(h);
    e = cudaStreamEndCapture(cap, &g);
  }
  h->stream = keep;
  h->timing = t;
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) return h->fail(PT_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  {
    // kernel launches per step: the kernel nodes of the captured graph
    size_t nn = 0;
    h->graph_kernels = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
      std::vector<cudaGraphNode_t> nodes(nn);
      if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
        for (auto nd : nodes) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++h->graph_kernels;
        }
    }
  }
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return h->fail(PT_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return PT_OK;
}

// ---------------------------------------------------------------- problem copy
int copy_problem(pt_tebd* h, const pt_chain_desc* chains, int n_chains, const pt_mpo_desc* mpos,
                 int n_mpos) {
  h->chains.resize(n_chains);
  for (int c = 0; c < n_chains; ++c) {
    const pt_chain_desc& d = chains[c];
    HostChain& hc = h->chains[c];
    if (d.N < 1) return h->fail(PT_ERR_ARG, "chain N must be >= 1");
    hc.N = d.N;
    const bool has_mps = d.gamma0 != nullptr;
    if (!has_mps && !d.rho0) return h->fail(PT_ERR_ARG, "chain needs rho0 or gamma0");
    if (d.N > 1 && (!d.gates_q || !d.gates_h)) return h->fail(PT_ERR_ARG, "chain needs gates");
    if (!has_mps) hc.rho0.assign((const cplx*)d.rho0, (const cplx*)d.rho0 + 4 * d.N);
    if (d.N > 1) {
      hc.gq.assign((const cplx*)d.gates_q, (const cplx*)d.gates_q + 256 * (d.N - 1));
      hc.gh.assign((const cplx*)d.gates_h, (const cplx*)d.gates_h + 256 * (d.N - 1));
    }
    if (d.local_prop) hc.local_prop.assign((const cplx*)d.local_prop, (const cplx*)d.local_prop + 16 * d.N);
    hc.mpo.assign(d.N, -1);
    if (d.ptmpo_id)
      for (int n = 0; n < d.N; ++n) {
        hc.mpo[n] = d.ptmpo_id[n];
        if (hc.mpo[n] >= n_mpos || hc.mpo[n] < -1) return h->fail(PT_ERR_ARG, "ptmpo_id out of range");
      }
    if (has_mps) {
      if (!d.chi0 || !d.kappa0 || !d.lambda0) return h->fail(PT_ERR_ARG, "gamma0 needs chi0, kappa0, lambda0");
      hc.chi0.assign(d.chi0, d.chi0 + d.N + 1);
      if (d.lognorm0) {
        hc.lognorm0.assign(d.lognorm0, d.lognorm0 + d.N + 1);
        for (double x : hc.lognorm0)
          if (!std::isfinite(x)) return h->fail(PT_ERR_ARG, "lognorm0 must be finite");
      }
      hc.kappa0.assign(d.kappa0, d.kappa0 + d.N);
      if (hc.chi0[0] != 1 || hc.chi0[d.N] != 1) return h->fail(PT_ERR_ARG, "chi0 ends must be 1");
      for (int n = 0; n < d.N; ++n) {
        if (hc.chi0[n] < 1 || hc.kappa0[n] < 1) return h->fail(PT_ERR_ARG, "chi0/kappa0 must be >= 1");
        size_t sz = (size_t)hc.chi0[n] * 4 * hc.kappa0[n] * hc.chi0[n + 1];
        hc.gamma0.emplace_back((const cplx*)d.gamma0[n], (const cplx*)d.gamma0[n] + sz);
      }
      for (int n = 0; n <= d.N; ++n)
        hc.lambda0.emplace_back(d.lambda0[n], d.lambda0[n] + hc.chi0[n]);
    }
  }
  h->mpos_in.resize(n_mpos);
  for (int m = 0; m < n_mpos; ++m) {
    const pt_mpo_desc& d = mpos[m];
    if (d.K < 1 || !d.kappa || !d.P) return h->fail(PT_ERR_ARG, "PT-MPO needs K >= 1, kappa, P");
    HostMpo& hm = h->mpos_in[m];
    hm.K = d.K;
    hm.kappa.assign(d.kappa, d.kappa + d.K + 1);
    for (int k = 0; k < d.K; ++k) {
      if (hm.kappa[k] < 1 || hm.kappa[k + 1] < 1) return h->fail(PT_ERR_ARG, "PT-MPO kappa must be >= 1");
      size_t sz = (size_t)hm.kappa[k] * 16 * hm.kappa[k + 1];
      hm.P.emplace_back((const cplx*)d.P[k], (const cplx*)d.P[k] + sz);
    }
  }
  return PT_OK;
}

// Fuse an on-site propagator LP (applied after P) into a PT-MPO: P~[a,p,p',b] = sum_q LP[p',q] P[a,p,q,b].
HostMpo fuse(const HostMpo& in, const cplx* LP) {
  HostMpo out = in;
  for (int k = 0; k < in.K; ++k) {
    const int ka = in.kappa[k], kb = in.kappa[k + 1];
    for (int a = 0; a < ka; ++a)
      for (int p = 0; p < 4; ++p)
        for (int pp = 0; pp < 4; ++pp)
          for (int b = 0; b < kb; ++b) {
            cplx s = 0;
            for (int q = 0; q < 4; ++q) s += LP[pp * 4 + q] * in.P[k][((size_t)(a * 4 + p) * 4 + q) * kb + b];
            out.P[k][((size_t)(a * 4 + p) * 4 + pp) * kb + b] = s;
          }
  }
  return out;
}

// ---------------------------------------------------------------- autotuner

// For each bond layer the kernels of two stages have candidates: the pivoted QR of the SVD (whole
// GPU / cluster shared memory / cluster global memory, as far as they fit) and the outer-block
// QR/LQ (whole GPU / one CTA per block). The tuner times every candidate once on a synthetic state
// at capacity (every Gamma and lambda at its capacity dims, seeded values), keeps the fastest, and
// caches the choice in a text file (one line per layer shape: key, QR route, outer-QR route,
// timings), keyed by GPU name, driver version, compute capability, precision and the layer's
// capacities. A layer whose key is cached is not timed again.
std::string tune_key(pt_tebd* h, const std::vector<BondWork>& v, int k_cap, int m_cap) {
  int dev = 0, drv = 0;
  cudaGetDevice(&dev);
  cudaDriverGetVersion(&drv);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  std::string name(prop.name);
  for (auto& ch : name)
    if (ch == ' ' || ch == '\t' || ch == '|') ch = '_';
  long long cols = 0;
  int mL = 0;
  for (auto& W : v) {
    cols += W.nL_cap + W.mR_cap;
    mL = std::max(mL, std::max(W.mL_cap, W.nR_cap));
  }
  char buf[512];
  snprintf(buf, sizeof buf, "%s|drv%d|sm%d%d|p%d|n%zu|k%d|m%d|c%lld|b%d", name.c_str(), drv, prop.major,
           prop.minor, (int)h->opt.precision, v.size(), k_cap, m_cap, cols, mL);
  return buf;
}

bool cache_lookup(const char* path, const std::string& key, int* qr, int* k2) {
  if (!path || !*path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[2048];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char* tab = strchr(line, '\t');
    if (!tab) continue;                                  // malformed: ignored
    if (std::string(line, tab - line) != key) continue;
    int a = -1, b = -1;
    if (sscanf(tab + 1, "%d\t%d", &a, &b) == 2 && a >= 0 && a <= 2 && b >= 0 && b <= 1) {
      *qr = a;                                           // the last valid line of a key wins
      *k2 = b;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, const pt_tebd::Route& r) {
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s\t%d\t%d\tms_qr=%.4f,%.4f,%.4f\tms_k2=%.4f,%.4f\n", key.c_str(), r.qr, r.k2, r.ms_qr[0],
          r.ms_qr[1], r.ms_qr[2], r.ms_k2[0], r.ms_k2[1]);
  fclose(f);
}

float time_once(pt_tebd* h, const std::function<void()>& launch) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, h->stream);
  launch();
  cudaEventRecord(b, h->stream);
  cudaEventSynchronize(b);
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

// the layer's route from the tune cache, if it holds one that fits
bool cached_route(pt_tebd* h, const BondWork* work, const std::vector<BondWork>& v, pt_tebd::Route& r) {
  const bool odd = work == h->d_odd;
  const int kc = odd ? h->kcap_odd : h->kcap_even, mc = odd ? h->mcap_odd : h->mcap_even;
  int qr = r.qr, k2 = r.k2;
  if (!cache_lookup(h->opt.tune_cache, tune_key(h, v, kc, mc), &qr, &k2)) return false;
  const bool qr_ok = qr == 2 || (qr == 1 && h->qr_smem_cluster > 0) || (qr == 0 && (odd ? h->qr_grid_odd : h->qr_grid_even));
  const bool k2_ok = k2 == 1 || (odd ? h->hqr_odd : h->hqr_even);
  if (!qr_ok || !k2_ok) return false;
  r.qr = qr;
  r.k2 = k2;
  r.cached = true;
  return true;
}

int tune_layer(pt_tebd* h, const BondWork* work, int n, const std::vector<BondWork>& v, pt_tebd::Route& r) {
  if (r.cached) return PT_OK;
  const bool odd = work == h->d_odd;
  const int kc = odd ? h->kcap_odd : h->kcap_even, mc = odd ? h->mcap_odd : h->mcap_even;
  const std::string key = tune_key(h, v, kc, mc);
  if (cached_route(h, work, v, r)) return PT_OK;     // another layer of the same shape was just timed
  cudaStream_t s = h->stream;
  // outer-block QR candidates (each on freshly built blocks; the faster of two runs)
  std::vector<int> k2c{1};
  if (odd ? h->hqr_odd : h->hqr_even) k2c.insert(k2c.begin(), 0);
  for (int c : k2c) {
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep)
      best = std::min(best, time_once(h, [&] {
                        ptk::k_build_blocks<<<dim3(h->gx_bond, n), 256, 0, s>>>(h->T, work, n);
                        enqueue_k2(h, work, n, c);
                      }));
    r.ms_k2[c] = best;
  }
  r.k2 = k2c[0];
  for (int c : k2c)
    if (r.ms_k2[c] < r.ms_k2[r.k2]) r.k2 = c;
  // D of the synthetic state, then the pivoted-QR candidates on it (a 128-reflector prefix each;
  // every candidate reads D and writes only its own workspace)
  if (!h->use_rsvd) {
    ptk::k_build_blocks<<<dim3(h->gx_bond, n), 256, 0, s>>>(h->T, work, n);
    enqueue_k2(h, work, n, r.k2);
    if (h->opt.precision == PT_FP64)
      ptk::k_theta_gate<<<dim3(h->gx_bond, n), 128, 0, s>>>(h->T, work, n);
    else
      ptk::launch_tc_theta(h->T, work, n, odd ? h->tiles_odd : h->tiles_even, (int)h->opt.precision, s);
  }
  std::vector<int> qrc{2};
  if (h->use_rsvd) qrc.clear();                      // the fast path's SVD has no pivoted QR
  else if (h->qr_smem_cluster > 0) qrc.insert(qrc.begin(), 1);
  if (!h->use_rsvd && (odd ? h->qr_grid_odd : h->qr_grid_even)) qrc.insert(qrc.begin(), 0);
  for (int c : qrc) {
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep)
      best = std::min(best, time_once(h, [&] { enqueue_qr(h, work, n, c, std::min(kc, 128)); }));
    r.ms_qr[c] = best;
  }
  if (!qrc.empty()) {
    r.qr = qrc[0];
    for (int c : qrc)
      if (r.ms_qr[c] < r.ms_qr[r.qr]) r.qr = c;
  }
  r.tuned = true;
  int rc = check_cuda(h, "autotune");
  if (rc == PT_OK) cache_store(h->opt.tune_cache, key, r);
  return rc;
}

// ---------------------------------------------------------------- initial state
// the log-norm carried per bond (the state is exp(sum) times the network): zero, or the caller's
std::vector<double> initial_lognorms(const pt_tebd* h) {
  std::vector<double> v(h->n_lams, 0.0);
  for (int c = 0; c < (int)h->chains.size(); ++c)
    for (size_t b = 0; b < h->chains[c].lognorm0.size(); ++b) v[h->lam0[c] + b] = h->chains[c].lognorm0[b];
  return v;
}

// Gamma and lambda of the initial augmented MPS (product state or the caller's gamma0/lambda0)
void upload_initial_gamma_lambda(pt_tebd* h) {
  for (int c = 0; c < (int)h->chains.size(); ++c) {
    HostChain& hc = h->chains[c];
    for (int n = 0; n < hc.N; ++n) {
      const int s = h->site0[c] + n;
      std::vector<cplx> g;
      if (hc.gamma0.empty()) g.assign(hc.rho0.begin() + 4 * n, hc.rho0.begin() + 4 * n + 4);
      else g = hc.gamma0[n];
      cudaMemcpyAsync(h->gam_a[s], g.data(), sizeof(cplx) * g.size(), cudaMemcpyHostToDevice, h->stream);
    }
    for (int b = 0; b <= hc.N; ++b) {
      const int B = h->lam0[c] + b;
      std::vector<double> l = hc.lambda0.empty() ? std::vector<double>{1.0} : hc.lambda0[b];
      cudaMemcpyAsync(h->lam_buf[B], l.data(), sizeof(double) * l.size(), cudaMemcpyHostToDevice, h->stream);
    }
  }
}

// the route of every layer: forced (tests), tuned (timed once, cached), or the default order; the
// tuning runs on a synthetic state at capacity, after which the initial state is restored
int choose_routes(pt_tebd* h, const std::vector<BondWork>& odd, const std::vector<BondWork>& even) {
  if (h->opt.force_route > 0) {
    const int qr = (h->opt.force_route - 1) % 4, k2 = (h->opt.force_route - 1) / 4;
    auto apply = [&](pt_tebd::Route& r, bool qr_grid, bool hqr) {
      const bool ok = (qr == 2 || (qr == 1 && h->qr_smem_cluster > 0) || (qr == 0 && qr_grid)) &&
                      (k2 == 1 || (k2 == 0 && hqr));
      if (ok) {
        r.qr = qr;
        r.k2 = k2;
      }
      return ok;
    };
    if (qr > 2 || k2 > 1 || !apply(h->route_odd, h->qr_grid_odd, h->hqr_odd) ||
        !apply(h->route_even, h->qr_grid_even, h->hqr_even))
      return h->fail(PT_ERR_ARG, "force_route: that route does not fit this problem");
    return PT_OK;
  }
  if (!h->opt.autotune || h->grid_blocks <= 0) return PT_OK;
  // layers the cache answers need no timing; the synthetic state only when one does
  const bool hit_odd = h->n_odd == 0 || cached_route(h, h->d_odd, odd, h->route_odd);
  const bool hit_even = h->n_even == 0 || cached_route(h, h->d_even, even, h->route_even);
  if (hit_odd && hit_even) return PT_OK;
  // synthetic state at capacity
  Tables& T = h->T;
  cudaMemcpyAsync(T.site_kappa, h->kcap_h.data(), sizeof(int) * h->n_sites, cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(T.lam_chi, h->lam_cap_h.data(), sizeof(int) * h->n_lams, cudaMemcpyHostToDevice, h->stream);
  ptk::k_tune_fill<<<4 * 152, 256, 0, h->stream>>>(T, h->n_sites, h->n_lams, 20220113u);
  int rc = check_cuda(h, "autotune fill");
  if (rc == PT_OK && h->n_odd > 0) rc = tune_layer(h, h->d_odd, h->n_odd, odd, h->route_odd);
  if (rc == PT_OK && h->n_even > 0) rc = tune_layer(h, h->d_even, h->n_even, even, h->route_even);
  // the synthetic run must not have tripped a device check; if it did, its timings are meaningless
  cudaMemcpyAsync(&h->tune_status, T.status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  if (h->tune_status != 0) {
    auto defaults = [&](pt_tebd::Route& r, bool qr_grid, bool hqr) {
      r.qr = qr_grid ? 0 : (h->qr_smem_cluster > 0 ? 1 : 2);
      r.k2 = hqr ? 0 : 1;
      r.tuned = false;
    };
    defaults(h->route_odd, h->qr_grid_odd, h->hqr_odd);
    defaults(h->route_even, h->qr_grid_even, h->hqr_even);
  }
  // back to the initial state
  upload_initial_gamma_lambda(h);
  cudaMemcpyAsync(T.site_kappa, h->kap_init_h.data(), sizeof(int) * h->n_sites, cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(T.lam_chi, h->chi_init_h.data(), sizeof(int) * h->n_lams, cudaMemcpyHostToDevice, h->stream);
  {
    const std::vector<double> ln = initial_lognorms(h);
    cudaMemcpyAsync(T.lam_lognorm, ln.data(), sizeof(double) * h->n_lams, cudaMemcpyHostToDevice, h->stream);
    cudaStreamSynchronize(h->stream);     // ln is a local host buffer
  }
  cudaMemsetAsync(T.step, 0, sizeof(int), h->stream);
  cudaMemsetAsync(T.status, 0, sizeof(int), h->stream);
  return rc != PT_OK ? rc : check_cuda(h, "autotune restore");
}

// ---------------------------------------------------------------- build the device state
int build(pt_tebd* h) {
  const int C = (int)h->chains.size();
  h->n_chains = C;
  // device PT-MPO list: the shared ones, then per-site fused copies where a local propagator is given
  std::vector<HostMpo> dm = h->mpos_in;
  std::vector<std::vector<int>> site_m(C);
  int K_limit = h->opt.max_steps > 0 ? h->opt.max_steps : 1024;
  bool any_mpo = false;
  for (int c = 0; c < C; ++c) {
    HostChain& hc = h->chains[c];
    site_m[c].assign(hc.N, -1);
    for (int n = 0; n < hc.N; ++n) {
      int m = hc.mpo[n];
      if (!hc.local_prop.empty()) {
        const cplx* LP = hc.local_prop.data() + 16 * n;
        HostMpo base;
        if (m >= 0) {
          base = h->mpos_in[m];
        } else {
          base.K = K_limit;
          base.kappa.assign(K_limit + 1, 1);
          std::vector<cplx> id(16, 0.0);
          for (int p = 0; p < 4; ++p) id[p * 4 + p] = 1.0;
          base.P.assign(K_limit, id);
        }
        dm.push_back(fuse(base, LP));
        m = (int)dm.size() - 1;
      }
      site_m[c][n] = m;
    }
  }
  for (int c = 0; c < C; ++c)
    for (int n = 0; n < h->chains[c].N; ++n)
      if (site_m[c][n] >= 0) {
        any_mpo = true;
        K_limit = std::min(K_limit, dm[site_m[c][n]].K);
      }
  if (!any_mpo) K_limit = h->opt.max_steps > 0 ? h->opt.max_steps : 1024;
  h->K_limit = K_limit;
  h->n_mpos = (int)dm.size();

  // layout and capacities
  h->site0.resize(C);
  h->lam0.resize(C);
  h->n_sites = 0;
  h->n_lams = 0;
  h->n_max = 0;
  for (int c = 0; c < C; ++c) {
    h->site0[c] = h->n_sites;
    h->lam0[c] = h->n_lams;
    h->n_sites += h->chains[c].N;
    h->n_lams += h->chains[c].N + 1;
    h->n_max = std::max(h->n_max, h->chains[c].N);
  }
  h->kcap_h.assign(h->n_sites, 1);
  h->site_mpo_h.assign(h->n_sites, -1);
  h->lam_cap_h.assign(h->n_lams, 1);
  h->site_cap_h.assign(h->n_sites, 0);
  std::vector<int>& kap_init = h->kap_init_h;
  std::vector<int>& chi_init = h->chi_init_h;
  kap_init.assign(h->n_sites, 1);
  chi_init.assign(h->n_lams, 1);
  const double BIG = 1e9;
  for (int c = 0; c < C; ++c) {
    HostChain& hc = h->chains[c];
    const int N = hc.N;
    for (int n = 0; n < N; ++n) {
      const int s = h->site0[c] + n;
      const int m = site_m[c][n];
      h->site_mpo_h[s] = m;
      int kc = 1;
      if (m >= 0)
        for (int k = 0; k <= dm[m].K; ++k) kc = std::max(kc, dm[m].kappa[k]);
      if (!hc.kappa0.empty()) {
        kc = std::max(kc, hc.kappa0[n]);
        kap_init[s] = hc.kappa0[n];
        if (m >= 0 && dm[m].kappa[0] != hc.kappa0[n])
          return h->fail(PT_ERR_ARG, "PT-MPO kappa[0] does not match the site's initial kappa");
      } else if (m >= 0 && dm[m].kappa[0] != 1) {
        return h->fail(PT_ERR_ARG, "PT-MPO kappa[0] must be 1 for a product initial state");
      }
      h->kcap_h[s] = kc;
    }
    // Liouville counting bound on each bond, capped at chi_max
    for (int b = 0; b <= N; ++b) {
      double L = 1, R = 1;
      for (int i = 0; i < b; ++i) L = std::min(BIG, L * 4.0 * h->kcap_h[h->site0[c] + i]);
      for (int i = b; i < N; ++i) R = std::min(BIG, R * 4.0 * h->kcap_h[h->site0[c] + i]);
      int cap = (int)std::min((double)h->opt.chi_max, std::min(L, R));
      if (b == 0 || b == N) cap = 1;
      if (!hc.chi0.empty()) {
        // chi_max caps every bond at every step, the initial augmented MPS included
        if (hc.chi0[b] > h->opt.chi_max)
          return h->fail(PT_ERR_CAPACITY, "initial MPS: bond " + std::to_string(b) + " of chain " +
                                              std::to_string(c) + " has chi0 = " + std::to_string(hc.chi0[b]) +
                                              " > chi_max = " + std::to_string(h->opt.chi_max));
        cap = std::max(cap, hc.chi0[b]);
        chi_init[h->lam0[c] + b] = hc.chi0[b];
      }
      h->lam_cap_h[h->lam0[c] + b] = std::max(1, cap);
    }
    for (int n = 0; n < N; ++n) {
      const int s = h->site0[c] + n, B = h->lam0[c] + n;
      h->site_cap_h[s] = (size_t)h->lam_cap_h[B] * 4 * h->kcap_h[s] * h->lam_cap_h[B + 1];
    }
  }

  // Gamma and lambda buffers
  h->gam_a.resize(h->n_sites);
  h->gam_b.resize(h->n_sites);
  for (int s = 0; s < h->n_sites; ++s) {
    h->gam_a[s] = (double2*)h->dalloc(sizeof(double2) * h->site_cap_h[s]);
    h->gam_b[s] = (double2*)h->dalloc(sizeof(double2) * h->site_cap_h[s]);
    if (!h->gam_a[s] || !h->gam_b[s]) return h->fail(PT_ERR_OOM, "Gamma buffers");
  }
  h->lam_buf.resize(h->n_lams);
  int maxchi = 1;
  for (int B = 0; B < h->n_lams; ++B) {
    h->lam_buf[B] = (double*)h->dalloc(sizeof(double) * h->lam_cap_h[B]);
    if (!h->lam_buf[B]) return h->fail(PT_ERR_OOM, "lambda buffers");
    maxchi = std::max(maxchi, h->lam_cap_h[B]);
  }
  // initial state
  upload_initial_gamma_lambda(h);

  // PT-MPOs and caps
  std::vector<int> mK(h->n_mpos), kap_off(h->n_mpos), P_off(h->n_mpos), cap_off(h->n_mpos);
  std::vector<int> kap_all;
  std::vector<const double2*> P_ptrs;
  std::vector<double2*> cap_ptrs;
  for (int m = 0; m < h->n_mpos; ++m) {
    mK[m] = dm[m].K;
    kap_off[m] = (int)kap_all.size();
    kap_all.insert(kap_all.end(), dm[m].kappa.begin(), dm[m].kappa.end());
    P_off[m] = (int)P_ptrs.size();
    size_t tot = 0;
    for (auto& p : dm[m].P) tot += p.size();
    double2* blob = (double2*)h->dalloc(sizeof(double2) * tot);
    if (!blob) return h->fail(PT_ERR_OOM, "PT-MPO tensors");
    size_t off = 0;
    for (auto& p : dm[m].P) {
      cudaMemcpyAsync(blob + off, p.data(), sizeof(cplx) * p.size(), cudaMemcpyHostToDevice, h->stream);
      P_ptrs.push_back(blob + off);
      off += p.size();
    }
    cap_off[m] = (int)cap_ptrs.size();
    int kmax = 1;
    for (int k : dm[m].kappa) kmax = std::max(kmax, k);
    double2* cb = (double2*)h->dalloc(sizeof(double2) * (size_t)(dm[m].K + 1) * kmax);
    if (!cb) return h->fail(PT_ERR_OOM, "caps");
    for (int k = 0; k <= dm[m].K; ++k) cap_ptrs.push_back(cb + (size_t)k * kmax);
  }

  // device tables
  Tables& T = h->T;
  std::vector<size_t> scap(h->site_cap_h);
  T.site_gam = upload(h, h->gam_a);
  T.site_alt = upload(h, h->gam_b);
  T.site_kappa = upload(h, kap_init);
  T.site_mpo = upload(h, h->site_mpo_h);
  T.site_cap = upload(h, scap);
  T.lam_ptr = upload(h, h->lam_buf);
  T.lam_chi = upload(h, chi_init);
  T.lam_cap = upload(h, h->lam_cap_h);
  T.lam_lognorm = upload(h, initial_lognorms(h));
  std::vector<int> Nv(C);
  for (int c = 0; c < C; ++c) Nv[c] = h->chains[c].N;
  T.chain_site0 = upload(h, h->site0);
  T.chain_lam0 = upload(h, h->lam0);
  T.chain_N = upload(h, Nv);
  std::vector<int> one{0};
  T.mpo_K = upload(h, mK.empty() ? one : mK);
  T.mpo_kappa_off = upload(h, kap_off.empty() ? one : kap_off);
  T.mpo_kappa = upload(h, kap_all.empty() ? one : kap_all);
  T.mpo_P_off = upload(h, P_off.empty() ? one : P_off);
  std::vector<const double2*> nullp{nullptr};
  T.mpo_P = upload(h, P_ptrs.empty() ? nullp : P_ptrs);
  T.mpo_cap_off = upload(h, cap_off.empty() ? one : cap_off);
  std::vector<double2*> nullc{nullptr};
  T.mpo_cap = upload(h, cap_ptrs.empty() ? nullc : cap_ptrs);
  T.step = upload(h, one);
  T.status = upload(h, one);
  if (!T.site_gam || !T.site_alt || !T.site_kappa || !T.site_mpo || !T.site_cap || !T.lam_ptr ||
      !T.lam_chi || !T.lam_cap || !T.lam_lognorm || !T.chain_site0 || !T.chain_lam0 ||
      !T.chain_N || !T.mpo_K || !T.mpo_kappa_off || !T.mpo_kappa || !T.mpo_P_off || !T.mpo_P ||
      !T.mpo_cap_off || !T.mpo_cap || !T.step || !T.status)
    return h->fail(PT_ERR_OOM, "device tables");
  if (h->n_mpos > 0) ptk::k_caps<<<h->n_mpos, 128, 0, h->stream>>>(T, h->n_mpos);

  // bond work lists (odd: 0-based bonds 0,2,..; even: 1,3,..) with private scratch
  std::vector<BondWork> odd, even;
  size_t max_bond_elems = 1;
  for (int c = 0; c < C; ++c) {
    HostChain& hc = h->chains[c];
    double2* gq = hc.N > 1 ? upload(h, (const double2*)hc.gq.data(), hc.gq.size()) : nullptr;
    double2* gh = hc.N > 1 ? upload(h, (const double2*)hc.gh.data(), hc.gh.size()) : nullptr;
    if (hc.N > 1 && (!gq || !gh)) return h->fail(PT_ERR_OOM, "gates");
    for (int b = 0; b + 1 < hc.N; ++b) {
      BondWork W{};
      W.chain = c;
      W.site_l = h->site0[c] + b;
      W.lam_l = h->lam0[c] + b;
      const bool is_odd = (b % 2) == 0;
      W.gate = (is_odd ? gq : gh) + 256 * b;
      const int sL = W.site_l, sR = sL + 1, BL = W.lam_l;
      const int chl = h->lam_cap_h[BL], chc = h->lam_cap_h[BL + 1], chr = h->lam_cap_h[BL + 2];
      W.mL_cap = chl * h->kcap_h[sL];
      W.nL_cap = 4 * chc;
      W.mR_cap = 4 * chc;
      W.nR_cap = h->kcap_h[sR] * chr;
      const int rL = std::min(W.mL_cap, W.nL_cap), rR = std::min(W.mR_cap, W.nR_cap);
      W.mD_cap = 4 * rL;
      W.nD_cap = 4 * rR;
      W.k_cap = std::min(W.mD_cap, W.nD_cap);
      size_t qls = (size_t)W.mL_cap * W.nL_cap, rls = (size_t)W.nL_cap * W.nL_cap;
      size_t qrs = (size_t)W.nR_cap * W.mR_cap, lrs = (size_t)W.mR_cap * W.mR_cap;
      size_t as = (size_t)W.mD_cap * W.nD_cap, vs = (size_t)W.k_cap * W.k_cap;
      W.QL = (double2*)h->dalloc(sizeof(double2) * qls);
      W.RL = (double2*)h->dalloc(sizeof(double2) * rls);
      W.QR = (double2*)h->dalloc(sizeof(double2) * qrs);
      W.LR = (double2*)h->dalloc(sizeof(double2) * lrs);
      W.HH = (double2*)h->dalloc(sizeof(double2) * (qls + qrs));
      W.A = (double2*)h->dalloc(sizeof(double2) * as);
      W.V = (double2*)h->dalloc(sizeof(double2) * vs);
      // sig and aux: singular values and the pivoted QR's column norms (k_cap), and the whole-GPU
      // outer-block QR's reflector scalars (n_L of B_L in aux, m_R of B_R^H in sig): on a chain's
      // edge bonds 4 chi_c exceeds k_cap
      const size_t sa = (size_t)std::max(W.k_cap, std::max(W.nL_cap, W.mR_cap));
      W.sig = (double*)h->dalloc(sizeof(double) * sa);
      W.aux = (double*)h->dalloc(sizeof(double) * sa);
      W.perm = (int*)h->dalloc(sizeof(int) * W.k_cap);
      W.info = (int*)h->dalloc(sizeof(int) * 16);
      if (!W.QL || !W.RL || !W.QR || !W.LR || !W.HH || !W.A || !W.V || !W.sig || !W.aux || !W.perm || !W.info)
        return h->fail(PT_ERR_OOM, "bond scratch");
      cudaMemsetAsync(W.info, 0, sizeof(int) * 16, h->stream);
      if (h->opt.precision != PT_FP64) {
        W.TA = h->dalloc(ptk::tc_pack_bytes(W, 0, (int)h->opt.precision));
        W.TB = h->dalloc(ptk::tc_pack_bytes(W, 1, (int)h->opt.precision));
        if (!W.TA || !W.TB) return h->fail(PT_ERR_OOM, "fast-path scratch");
      }
      if (h->opt.precision == PT_BF16_OZAKI) {
        // the randomized truncated SVD: l <= chi_max + oversampling columns
        W.rs_mx = std::max(W.mD_cap, W.nD_cap);
        W.L_cap = std::max(1, std::min(W.k_cap, h->opt.chi_max + ptk::RSVD_OVERSAMPLE));
        const size_t L = (size_t)W.L_cap;
        W.RY = (double2*)h->dalloc(sizeof(double2) * W.rs_mx * L);
        W.RZ = (double2*)h->dalloc(sizeof(double2) * W.k_cap * L);
        W.RH = (double2*)h->dalloc(sizeof(double2) * W.rs_mx * L);
        W.RR = (double2*)h->dalloc(sizeof(double2) * L * L);
        W.Rtau = (double*)h->dalloc(sizeof(double) * L);
        W.ZA = (unsigned char*)h->dalloc(ptk::zgemm_pack_bytes(W.rs_mx, W.rs_mx, 0));
        W.ZA2 = (unsigned char*)h->dalloc(ptk::zgemm_pack_bytes(W.rs_mx, W.rs_mx, 0));
        // B operands: up to L_cap columns with K up to rs_mx, or (the residual D - Q Z^H) up to
        // rs_mx columns with K up to L_cap
        W.ZB = (unsigned char*)h->dalloc(std::max(ptk::zgemm_pack_bytes(W.L_cap, W.rs_mx, 1),
                                                  ptk::zgemm_pack_bytes(W.rs_mx, W.L_cap, 1)));
        if (!W.RY || !W.RZ || !W.RH || !W.RR || !W.Rtau || !W.ZA || !W.ZA2 || !W.ZB)
          return h->fail(PT_ERR_OOM, "fast-path SVD scratch");
      }
      {
        const size_t ma = (size_t)std::max(W.mD_cap, W.nD_cap);
        W.G64 = (double2*)h->dalloc(sizeof(double2) * vs);
        W.Y64 = (double2*)h->dalloc(sizeof(double2) * ma * W.k_cap);
        W.qperm = (int*)h->dalloc(sizeof(int) * W.k_cap);
        if (!W.G64 || !W.Y64 || !W.qperm) return h->fail(PT_ERR_OOM, "SVD scratch");
      }
      if (W.nL_cap > 2048 || W.mR_cap > 2048)
        return h->fail(PT_ERR_CAPACITY, "QR reduction supports at most 2048 columns (4 chi <= 2048)");
      max_bond_elems = std::max(max_bond_elems, std::max(qls + qrs, as));
      (is_odd ? odd : even).push_back(W);
    }
  }
  h->n_odd = (int)odd.size();
  h->n_even = (int)even.size();
  for (auto& W : odd) h->bond_info.push_back(W.info);
  for (auto& W : even) h->bond_info.push_back(W.info);
  // cluster size: about 8 column pairs per CTA of 32 warps, at most 16 CTAs per matrix
  auto pick = [&](const std::vector<BondWork>& v) {
    int k = 1;
    for (auto& W : v) k = std::max(k, W.k_cap);
    return ptk::jacobi_cluster_size(std::max(1, std::min(16, (k / 2 + 7) / 8)));
  };
  h->cl_odd = pick(odd);
  h->cl_even = pick(even);
  if (h->opt.precision != PT_FP64) {
    auto tiles = [&](const std::vector<BondWork>& v) {
      long long t = 0;
      for (auto& W : v) t += ptk::tc_tile_cap(W, (int)h->opt.precision);
      return (int)std::min<long long>(t, 1 << 30);
    };
    h->tiles_odd = tiles(odd);
    h->tiles_even = tiles(even);
  }
  {
    auto dims = [&](const std::vector<BondWork>& v, int* kc, int* mc) {
      for (auto& W : v) {
        *kc = std::max(*kc, W.k_cap);
        *mc = std::max(*mc, std::max(W.mD_cap, W.nD_cap));
      }
    };
    dims(odd, &h->kcap_odd, &h->mcap_odd);
    dims(even, &h->kcap_even, &h->mcap_even);
    int k = std::max(h->kcap_odd, h->kcap_even);
    h->qr_cluster = ptk::qrcp_cluster_size(std::max(1, std::min(16, (k + 31) / 32)),
                                           std::max(h->mcap_odd, h->mcap_even), k);
    h->qr_smem_cluster = ptk::qrcp_smem_cluster(std::max(h->mcap_odd, h->mcap_even), k);
  }
  // bond SVDs: the whole-GPU cooperative kernels when the device can co-schedule them, else one
  // thread-block cluster per matrix
  h->grid_blocks = std::max(h->n_odd, h->n_even) <= 1024 ? ptk::jacobi_grid_blocks() : 0;
  {
    // which kernels fit each layer: the whole-GPU pivoted QR where the layer's columns fit one per
    // warp; the cluster shared-memory one where a matrix fits 200 KB per CTA; the global-memory one
    // always; the whole-GPU outer-block QR where every block's columns fit the CTAs' share
    const bool ok = h->grid_blocks > 0 && ptk::qrcp_grid_ok();
    auto fits = [&](const std::vector<BondWork>& v, int mc) {
      int tot = 0;
      for (auto& W : v) tot += W.k_cap;
      return ok && !v.empty() && ptk::qrcp_grid_fits((int)v.size(), mc, tot, h->grid_blocks);
    };
    h->qr_grid_odd = fits(odd, h->mcap_odd);
    h->qr_grid_even = fits(even, h->mcap_even);
    // the outer-block reductions: whole GPU when every block's columns fit the CTAs' share
    const bool hok = h->grid_blocks > 0 && ptk::hqr_grid_ok();
    auto hfits = [&](const std::vector<BondWork>& v) {
      long long cols = 0;
      for (auto& W : v) cols += W.nL_cap + W.mR_cap;
      return hok && !v.empty() && cols < (1LL << 30) &&
             ptk::hqr_grid_fits((int)cols, 2 * (int)v.size(), h->grid_blocks);
    };
    h->hqr_odd = hfits(odd);
    h->hqr_even = hfits(even);
    // default order (no tuning): whole GPU, then cluster shared memory, then cluster global memory
    auto defaults = [&](pt_tebd::Route& r, bool qr_grid, bool hqr) {
      r.qr = qr_grid ? 0 : (h->qr_smem_cluster > 0 ? 1 : 2);
      r.k2 = hqr ? 0 : 1;
    };
    defaults(h->route_odd, h->qr_grid_odd, h->hqr_odd);
    defaults(h->route_even, h->qr_grid_even, h->hqr_even);
  }
  if (h->opt.precision == PT_BF16_OZAKI && h->grid_blocks > 0 && ptk::hqr_items_ok()) {
    // the fast path's randomized truncated SVD: item lists per layer, the sketch matrix
    auto lists = [&](const std::vector<BondWork>& v, ptk::RsvdLists& L) {
      const int n = std::max<int>(1, (int)v.size());
      long long cols = 0, tiles = 0;
      L.m_cap = L.l_cap = 1;
      for (auto& W : v) {
        cols += W.L_cap;
        tiles += ptk::zgemm_tile_cap(W.rs_mx, W.L_cap);
        L.m_cap = std::max(L.m_cap, W.rs_mx);
        L.l_cap = std::max(L.l_cap, W.L_cap);
      }
      L.tile_cap = (int)std::min<long long>(tiles, 1 << 30);
      ptk::ZGemmItem** z[7] = {&L.gy1, &L.gz1, &L.gy2, &L.gz2, &L.gres, &L.gu, &L.gv};
      for (auto p : z) *p = (ptk::ZGemmItem*)h->dalloc(sizeof(ptk::ZGemmItem) * n);
      ptk::QRItem** q[4] = {&L.q1, &L.qz, &L.q2, &L.qb};
      for (auto p : q) *p = (ptk::QRItem*)h->dalloc(sizeof(ptk::QRItem) * n);
      L.fro_part = (double*)h->dalloc(sizeof(double) * n * ptk::RSVD_FRO_PARTS);
      bool ok = L.fro_part != nullptr;
      for (auto p : z) ok = ok && *p;
      for (auto p : q) ok = ok && *p;
      return ok && cols <= (long long)h->grid_blocks * 384;
    };
    bool ok = lists(odd, h->rs_odd) && lists(even, h->rs_even);
    int rows = 1, cols = 1;
    for (auto* v : {&odd, &even})
      for (auto& W : *v) {
        rows = std::max(rows, W.k_cap);
        cols = std::max(cols, W.L_cap);
      }
    h->ld_omega = rows;
    h->d_omega = (double2*)h->dalloc(sizeof(double2) * (size_t)rows * cols);
    if (!h->d_omega) return h->fail(PT_ERR_OOM, "fast-path sketch matrix");
    ptk::launch_rsvd_omega(h->d_omega, rows, cols, 20220113u, h->stream);
    h->use_rsvd = ok;
  }
  h->d_sync3 = (unsigned*)h->dalloc(sizeof(unsigned) * 4);
  h->d_cnt_odd = (int*)h->dalloc(sizeof(int) * 2 * std::max(1, h->n_odd));
  h->d_cnt_even = (int*)h->dalloc(sizeof(int) * 2 * std::max(1, h->n_even));
  if (!h->d_sync3 || !h->d_cnt_odd || !h->d_cnt_even) return h->fail(PT_ERR_OOM, "Jacobi barrier state");
  cudaMemsetAsync(h->d_sync3, 0, sizeof(unsigned) * 4, h->stream);
  h->d_odd = odd.empty() ? nullptr : upload(h, odd);
  h->d_even = even.empty() ? nullptr : upload(h, even);
  h->gx_bond = (int)std::min<size_t>(256, (max_bond_elems + 255) / 256);

  if (h->use_rsvd) {
    // the fast path's Gamma recovery on the tensor cores: per bond a left item (Q_L times U, C in HH)
    // and a right item (Q_R^H times V, C in HH + mL_cap nL_cap), packed planes at capacity
    auto rec_list = [&](const std::vector<BondWork>& v, pt_tebd::RecList& R) -> int {
      if (v.empty() || 2 * (int)v.size() > ptk::zgemm_max_items()) return PT_OK;
      std::vector<ptk::ZGemmItem> items(2 * v.size());
      std::vector<int*> bc(v.size());
      long long tiles = 0;
      for (size_t w = 0; w < v.size(); ++w) {
        const BondWork& W = v[w];
        bc[w] = (int*)h->dalloc(sizeof(int) * (size_t)(W.nL_cap + W.mR_cap));
        if (!bc[w]) return h->fail(PT_ERR_OOM, "tensor-core recovery column maps");
        for (int side = 0; side < 2; ++side) {
          ptk::ZGemmItem& it = items[2 * w + side];
          it = ptk::ZGemmItem{};
          it.cap_m = side == 0 ? W.mL_cap : W.nR_cap;
          it.cap_k = side == 0 ? std::min(W.mL_cap, W.nL_cap) : std::min(W.nR_cap, W.mR_cap);
          it.cap_n = side == 0 ? W.nL_cap : W.mR_cap;
          it.opA = ptk::ZOP_N;
          it.opB = side == 0 ? ptk::ZOP_T : ptk::ZOP_N;
          it.bcol = side == 0 ? bc[w] : bc[w] + W.nL_cap;
          it.C = side == 0 ? W.HH : W.HH + (size_t)W.mL_cap * W.nL_cap;
          it.TA = (unsigned char*)h->dalloc(ptk::zgemm_pack_bytes(it.cap_m, it.cap_k, 0));
          it.TB = (unsigned char*)h->dalloc(ptk::zgemm_pack_bytes(it.cap_n, it.cap_k, 1));
          if (!it.TA || !it.TB) return h->fail(PT_ERR_OOM, "tensor-core recovery scratch");
          tiles += ptk::zgemm_tile_cap(it.cap_m, it.cap_n);
          R.mcap = std::max(R.mcap, it.cap_m);
          R.ncap = std::max(R.ncap, it.cap_n);
        }
      }
      R.tile_cap = (int)std::min<long long>(tiles, 1 << 30);
      R.items = upload(h, items);
      R.bcols = upload(h, bc);
      if (!R.items || !R.bcols) return h->fail(PT_ERR_OOM, "tensor-core recovery items");
      return PT_OK;
    };
    int rc = rec_list(odd, h->rec_odd);
    if (rc == PT_OK) rc = rec_list(even, h->rec_even);
    if (rc != PT_OK) return rc;
  }

  // site work list
  std::vector<SiteWork> sw;
  size_t max_site = 1;
  for (int c = 0; c < C; ++c)
    for (int n = 0; n < h->chains[c].N; ++n) {
      const int s = h->site0[c] + n;
      if (h->site_mpo_h[s] < 0) continue;
      sw.push_back({s, h->site_mpo_h[s], h->lam0[c] + n, 0});
      max_site = std::max(max_site, h->site_cap_h[s]);
    }
  h->n_site_work = (int)sw.size();
  h->d_sites = sw.empty() ? nullptr : upload(h, sw);
  h->gx_site = (int)std::min<size_t>(256, (max_site + 255) / 256);
  if (h->opt.precision == PT_BF16_OZAKI && h->use_rsvd && !sw.empty() && h->n_site_work <= ptk::zgemm_max_items()) {
    // the fast path's site layer on the tensor cores: per site the GEMM's output scratch and the
    // packed slice planes of both operands at capacity; live fields are written by the plan kernel
    std::vector<ptk::ZGemmItem> items(sw.size());
    long long tiles = 0;
    for (size_t w = 0; w < sw.size(); ++w) {
      const int s = sw[w].site, B = sw[w].lam;
      ptk::ZGemmItem& it = items[w];
      it = ptk::ZGemmItem{};
      it.cap_m = h->lam_cap_h[B] * h->lam_cap_h[B + 1];
      it.cap_k = it.cap_n = 4 * h->kcap_h[s];
      it.opA = ptk::ZOP_N;
      it.opB = ptk::ZOP_T;
      it.C = (double2*)h->dalloc(sizeof(double2) * std::max(h->site_cap_h[s], (size_t)it.cap_m * it.cap_n));
      it.TA = (unsigned char*)h->dalloc(ptk::zgemm_pack_bytes(it.cap_m, it.cap_k, 0));
      it.TB = (unsigned char*)h->dalloc(ptk::zgemm_pack_bytes(it.cap_n, it.cap_k, 1));
      if (!it.C || !it.TA || !it.TB) return h->fail(PT_ERR_OOM, "tensor-core site contraction scratch");
      tiles += ptk::zgemm_tile_cap(it.cap_m, it.cap_n);
      h->site_mcap = std::max(h->site_mcap, it.cap_m);
      h->site_ncap = std::max(h->site_ncap, it.cap_n);
    }
    h->site_tile_cap = (int)std::min<long long>(tiles, 1 << 30);
    h->d_site_items = upload(h, items);
    if (!h->d_site_items) return h->fail(PT_ERR_OOM, "tensor-core site contraction items");
  }

  // readout buffers
  h->ld = maxchi;
  h->d_Lbuf = (double2*)h->dalloc(sizeof(double2) * (size_t)C * (h->n_max + 1) * h->ld);
  h->d_Rbuf = (double2*)h->dalloc(sizeof(double2) * (size_t)C * (h->n_max + 1) * h->ld);
  h->d_ops_now = (double2*)h->dalloc(sizeof(double2) * 4 * pt_tebd::MAX_OPS);
  h->d_obs_now = (double2*)h->dalloc(sizeof(double2) * (size_t)C * h->n_max * pt_tebd::MAX_OPS);
  h->d_tr_now = (double2*)h->dalloc(sizeof(double2) * C);
  h->hist_cap = h->K_limit + 1;
  h->blog_nb = std::max(1, std::max(h->n_odd, h->n_even));
  {
    const size_t nlog = (size_t)h->hist_cap * 6 * h->blog_nb * ptk::BOND_LOG_INTS;
    h->d_blog = (int*)h->dalloc(sizeof(int) * nlog);
    if (!h->d_blog) return h->fail(PT_ERR_OOM, "bond log");
    cudaMemsetAsync(h->d_blog, 0, sizeof(int) * nlog, h->stream);
  }
  if (!h->d_Lbuf || !h->d_Rbuf || !h->d_ops_now || !h->d_obs_now || !h->d_tr_now)
    return h->fail(PT_ERR_OOM, "readout buffers");
  {
    // M_n capacity per site: chi_l,cap x 4 x chi_r,cap (the augmented leg is closed)
    std::vector<size_t> moff(h->n_sites, 0);
    size_t tot = 0, mx = 1;
    for (int c = 0; c < C; ++c)
      for (int n = 0; n < h->chains[c].N; ++n) {
        const int s = h->site0[c] + n, B = h->lam0[c] + n;
        const size_t cap = (size_t)h->lam_cap_h[B] * 4 * h->lam_cap_h[B + 1];
        moff[s] = tot;
        tot += cap;
        mx = std::max(mx, cap);
      }
    h->d_Mbuf = (double2*)h->dalloc(sizeof(double2) * std::max<size_t>(1, tot));
    h->d_moff = upload(h, moff);
    if (!h->d_Mbuf || !h->d_moff) return h->fail(PT_ERR_OOM, "readout buffers");
    h->gx_m = (int)std::min<size_t>(64, (mx + 255) / 256);
  }
  {
    const int rc = choose_routes(h, odd, even);
    if (rc != PT_OK) return rc;
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return check_cuda(h, "init");
  return check_cuda(h, "init");
}

void op_vectors(const double* ops, int n_ops, std::vector<cplx>& out) {
  // vec(O^T)[i*2+j] = O[j][i]
  out.resize(4 * (size_t)n_ops);
  const cplx* O = (const cplx*)ops;
  for (int k = 0; k < n_ops; ++k)
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) out[4 * k + i * 2 + j] = O[4 * k + j * 2 + i];
}

}  // namespace

namespace ptk {
void set_global_error(const char* msg) { g_err = msg; }
}  // namespace ptk

// ==================================================================== C ABI
extern "C" {

void pt_tebd_set_allocator(pt_alloc_fn alloc, pt_free_fn free_fn, void* ctx) {
  g_alloc = alloc;
  g_free = free_fn;
  g_ctx = ctx;
}

const char* pt_tebd_last_error(pt_tebd_t h) { return h ? h->err.c_str() : g_err.c_str(); }

int pt_tebd_init(pt_tebd_t* out, const pt_chain_desc* chains, int n_chains, const pt_mpo_desc* mpos,
                 int n_mpos, const pt_options* opt, void* cuda_stream) {
  if (!out || !chains || n_chains < 1 || !opt || (n_mpos > 0 && !mpos) || n_mpos < 0) {
    g_err = "pt_tebd_init: bad arguments";
    return PT_ERR_ARG;
  }
  *out = nullptr;
  NvtxRange nv("pt_tebd_init");
  pt_tebd* h = new pt_tebd();
  h->stream = (cudaStream_t)cuda_stream;
  h->opt = *opt;
  if (h->opt.chi_max < 1 || !(h->opt.eps >= 0.0) || h->opt.multiplet_tol < 0.0) {
    h->fail(PT_ERR_ARG, "pt_tebd_init: chi_max >= 1, eps >= 0, multiplet_tol >= 0 required");
    delete h;
    return PT_ERR_ARG;
  }
  if (h->opt.max_sweeps <= 0) h->opt.max_sweeps = 60;
  if (h->opt.precision < PT_FP64 || h->opt.precision > PT_BF16_OZAKI) {
    h->fail(PT_ERR_ARG, "pt_tebd_init: unknown precision");
    delete h;
    return PT_ERR_ARG;
  }
  int rc = copy_problem(h, chains, n_chains, mpos, n_mpos);
  if (rc == PT_OK) rc = build(h);
  if (rc == PT_OK && h->opt.use_graph) rc = capture_graph(h);
  if (rc != PT_OK) {
    g_err = h->err;
    h->release();
    delete h;
    return rc;
  }
  *out = h;
  return PT_OK;
}

int pt_tebd_set_observables(pt_tebd_t h, const double* ops, int n_ops) {
  if (!h || n_ops < 0 || n_ops > pt_tebd::MAX_OPS || (n_ops > 0 && !ops))
    return h ? h->fail(PT_ERR_ARG, "set_observables: 0 <= n_ops <= 16") : PT_ERR_ARG;
  std::vector<cplx> v;
  op_vectors(ops, n_ops, v);
  if (!h->d_ops) {
    h->d_ops = (double2*)h->dalloc(sizeof(double2) * 4 * pt_tebd::MAX_OPS);
    if (!h->d_ops) return h->fail(PT_ERR_OOM, "ops");
  }
  if (h->d_hist && h->n_ops != n_ops) return h->fail(PT_ERR_ARG, "set_observables: op count is fixed once set");
  if (!h->d_hist && n_ops > 0) {
    const size_t n = (size_t)h->hist_cap * h->n_chains * h->n_max * n_ops;
    h->d_hist = (double2*)h->dalloc(sizeof(double2) * n);
    h->d_hist_tr = (double2*)h->dalloc(sizeof(double2) * (size_t)h->hist_cap * h->n_chains);
    if (!h->d_hist || !h->d_hist_tr) return h->fail(PT_ERR_OOM, "history");
    cudaMemsetAsync(h->d_hist, 0, sizeof(double2) * n, h->stream);
    cudaMemsetAsync(h->d_hist_tr, 0, sizeof(double2) * (size_t)h->hist_cap * h->n_chains, h->stream);
  }
  if (n_ops > 0) cudaMemcpyAsync(h->d_ops, v.data(), sizeof(cplx) * v.size(), cudaMemcpyHostToDevice, h->stream);
  h->n_ops = n_ops;
  // record the current step, and re-capture the step graph so it includes the readout
  enqueue_observe_history(h);
  int rc = check_cuda(h, "set_observables");
  if (rc == PT_OK && h->opt.use_graph) rc = capture_graph(h);
  return rc;
}

int pt_tebd_step(pt_tebd_t h, int n_steps) {
  if (!h || n_steps < 0) return PT_ERR_ARG;
  if (h->steps_done + n_steps > h->K_limit)
    return h->fail(PT_ERR_STEPS, "step: past the end of the PT-MPOs / history capacity");
  h->ev_used = 0;
  NvtxRange nv("pt_tebd_step");
  for (int i = 0; i < n_steps; ++i) {
    if (h->graph && !h->timing) {
      if (cudaGraphLaunch(h->graph, h->stream) != cudaSuccess) return check_cuda(h, "graph launch");
    } else {
      enqueue_step(h);
    }
  }
  h->steps_done += n_steps;
  if (h->timing) {
    cudaStreamSynchronize(h->stream);
    for (int k = 0; k < 9; ++k) h->stage_ms[k] = 0;
    for (size_t i = 0; i < h->ev_used; ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, h->ev[i].second.first, h->ev[i].second.second);
      h->stage_ms[h->ev[i].first] += ms;
    }
  }
  return check_cuda(h, "step");
}

int pt_tebd_sync(pt_tebd_t h) {
  if (!h) return PT_ERR_ARG;
  int rc = check_cuda(h, "sync");
  if (rc != PT_OK) return rc;
  return read_status(h);
}

int pt_tebd_observe(pt_tebd_t h, const double* ops, int n_ops, double* out, double* trace_out,
                    int normalize) {
  if (!h || n_ops < 0 || n_ops > pt_tebd::MAX_OPS || (n_ops > 0 && (!ops || !out))) return PT_ERR_ARG;
  std::vector<cplx> v;
  op_vectors(ops, n_ops, v);
  if (n_ops > 0) cudaMemcpyAsync(h->d_ops_now, v.data(), sizeof(cplx) * v.size(), cudaMemcpyHostToDevice, h->stream);
  ptk::k_observe_m<<<dim3(h->gx_m, h->n_chains, h->n_max), 256, 0, h->stream>>>(h->T, h->n_chains, h->d_Mbuf,
                                                                                  h->d_moff);
  ptk::k_observe<<<h->n_chains, 256, 0, h->stream>>>(h->T, h->n_chains, h->d_ops_now, n_ops, h->n_max,
                                                     h->d_obs_now, h->d_tr_now, h->d_Lbuf, h->d_Rbuf,
                                                     h->ld, 0, h->d_Mbuf, h->d_moff);
  int rc = check_cuda(h, "observe");
  if (rc != PT_OK) return rc;
  const size_t n = (size_t)h->n_chains * h->n_max * n_ops;
  std::vector<cplx> o(n), tr(h->n_chains);
  cudaMemcpyAsync(o.data(), h->d_obs_now, sizeof(cplx) * n, cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(tr.data(), h->d_tr_now, sizeof(cplx) * h->n_chains, cudaMemcpyDeviceToHost, h->stream);
  rc = read_status(h);
  if (rc != PT_OK) return rc;
  for (int c = 0; c < h->n_chains; ++c) {
    const cplx t = tr[c];
    for (size_t i = 0; i < (size_t)h->n_max * n_ops; ++i) {
      cplx x = o[(size_t)c * h->n_max * n_ops + i];
      if (normalize) x /= t;
      ((cplx*)out)[(size_t)c * h->n_max * n_ops + i] = x;
    }
  }
  if (trace_out) std::memcpy(trace_out, tr.data(), sizeof(cplx) * h->n_chains);
  return PT_OK;
}

int pt_tebd_read_history(pt_tebd_t h, int first, int count, double* out, double* trace_out) {
  if (!h || first < 0 || count < 0 || first + count > h->hist_cap || !h->d_hist) return PT_ERR_ARG;
  const size_t per = (size_t)h->n_chains * h->n_max * h->n_ops;
  if (out)
    cudaMemcpyAsync(out, h->d_hist + (size_t)first * per, sizeof(cplx) * per * count, cudaMemcpyDeviceToHost,
                    h->stream);
  if (trace_out)
    cudaMemcpyAsync(trace_out, h->d_hist_tr + (size_t)first * h->n_chains, sizeof(cplx) * h->n_chains * count,
                    cudaMemcpyDeviceToHost, h->stream);
  return read_status(h);
}

int pt_tebd_read_bond_log(pt_tebd_t h, int first, int count, int* out, size_t cap_ints) {
  if (!h || first < 0 || count < 0 || first + count > h->hist_cap || (count > 0 && !out)) return PT_ERR_ARG;
  const size_t per = (size_t)6 * h->blog_nb * ptk::BOND_LOG_INTS;
  if ((size_t)count * per > cap_ints) return h->fail(PT_ERR_ARG, "read_bond_log: output buffer too small");
  if (count > 0)
    cudaMemcpyAsync(out, h->d_blog + (size_t)first * per, sizeof(int) * per * count, cudaMemcpyDeviceToHost,
                    h->stream);
  // a diagnostic: readable after a device error (the log shows which bond raised it), so only a
  // CUDA error fails here
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return check_cuda(h, "read_bond_log");
  return h->blog_nb;
}

int pt_tebd_apply_local(pt_tebd_t h, int chain, int site, const double* op2x2, int side) {
  if (!h || chain < 0 || chain >= h->n_chains || site < 0 || site >= h->chains[chain].N || !op2x2 ||
      (side != 0 && side != 1))
    return h ? h->fail(PT_ERR_ARG, "apply_local: bad arguments") : PT_ERR_ARG;
  const cplx* A = (const cplx*)op2x2;
  cplx S[16];
  // left: S = A (x) I ; right: S = I (x) A^T, in vec index p = i*2 + j
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l) {
          const int p = i * 2 + j, q = k * 2 + l;
          cplx v = 0;
          if (side == 0) v = (j == l) ? A[i * 2 + k] : 0.0;
          else v = (i == k) ? A[l * 2 + j] : 0.0;
          S[p * 4 + q] = v;
        }
  ptk::launch_apply_local(h->T, h->site0[chain] + site, h->lam0[chain] + site, (const double2*)S, h->stream);
  return check_cuda(h, "apply_local");
}

int pt_tebd_steps_done(pt_tebd_t h) { return h ? h->steps_done : PT_ERR_ARG; }

int pt_tebd_get_routes(pt_tebd_t h, int* out8, float* ms10) {
  if (!h || !out8) return PT_ERR_ARG;
  const pt_tebd::Route* r[2] = {&h->route_odd, &h->route_even};
  for (int l = 0; l < 2; ++l) {
    out8[4 * l + 0] = r[l]->qr;
    out8[4 * l + 1] = r[l]->k2;
    out8[4 * l + 2] = r[l]->tuned ? 1 : 0;
    out8[4 * l + 3] = r[l]->cached ? 1 : 0;
    if (ms10) {
      for (int i = 0; i < 3; ++i) ms10[5 * l + i] = r[l]->ms_qr[i];
      for (int i = 0; i < 2; ++i) ms10[5 * l + 3 + i] = r[l]->ms_k2[i];
    }
  }
  return PT_OK;
}

int pt_tune_cache_lookup(const char* path, const char* key, int* qr, int* k2) {
  if (!path || !key || !qr || !k2) return PT_ERR_ARG;
  return cache_lookup(path, key, qr, k2) ? 1 : 0;
}

int pt_tune_cache_store(const char* path, const char* key, int qr, int k2) {
  if (!path || !key || qr < 0 || qr > 2 || k2 < 0 || k2 > 1 || strchr(key, '\t') || strchr(key, '\n'))
    return PT_ERR_ARG;
  pt_tebd::Route r;
  r.qr = qr;
  r.k2 = k2;
  cache_store(path, key, r);
  return PT_OK;
}

int pt_tebd_step_kernels(pt_tebd_t h) {
  if (!h) return PT_ERR_ARG;
  if (!h->graph) return h->fail(PT_ERR_ARG, "step_kernels: the handle has no captured step graph");
  return h->graph_kernels;
}

int pt_tebd_get_dims(pt_tebd_t h, int chain, int* chi, int* kappa) {
  if (!h || chain < 0 || chain >= h->n_chains) return PT_ERR_ARG;
  const int N = h->chains[chain].N;
  if (chi) cudaMemcpyAsync(chi, h->T.lam_chi + h->lam0[chain], sizeof(int) * (N + 1), cudaMemcpyDeviceToHost, h->stream);
  if (kappa) cudaMemcpyAsync(kappa, h->T.site_kappa + h->site0[chain], sizeof(int) * N, cudaMemcpyDeviceToHost, h->stream);
  return read_status(h);
}

int pt_tebd_get_lambda(pt_tebd_t h, int chain, int bond, double* out, int cap) {
  if (!h || chain < 0 || chain >= h->n_chains || bond < 0 || bond > h->chains[chain].N || !out) return PT_ERR_ARG;
  const int B = h->lam0[chain] + bond;
  int chi = 0;
  cudaMemcpyAsync(&chi, h->T.lam_chi + B, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  const int n = std::min(chi, cap);
  cudaMemcpyAsync(out, h->lam_buf[B], sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
  int rc = read_status(h);
  return rc == PT_OK ? chi : rc;
}

int pt_tebd_get_lognorm(pt_tebd_t h, int chain, double* out) {
  if (!h || chain < 0 || chain >= h->n_chains || !out) return PT_ERR_ARG;
  const int N = h->chains[chain].N;
  std::vector<double> v(N + 1);
  cudaMemcpyAsync(v.data(), h->T.lam_lognorm + h->lam0[chain], sizeof(double) * (N + 1), cudaMemcpyDeviceToHost,
                  h->stream);
  int rc = read_status(h);
  double s = 0;
  for (double x : v) s += x;
  *out = s;
  return rc;
}

int pt_tebd_get_lognorms(pt_tebd_t h, int chain, double* out) {
  if (!h || chain < 0 || chain >= h->n_chains || !out) return PT_ERR_ARG;
  const int N = h->chains[chain].N;
  cudaMemcpyAsync(out, h->T.lam_lognorm + h->lam0[chain], sizeof(double) * (N + 1), cudaMemcpyDeviceToHost,
                  h->stream);
  return read_status(h);
}

int pt_tebd_get_gamma(pt_tebd_t h, int chain, int site, double* out, size_t cap) {
  if (!h || chain < 0 || chain >= h->n_chains || site < 0 || site >= h->chains[chain].N) return PT_ERR_ARG;
  const int s = h->site0[chain] + site, B = h->lam0[chain] + site;
  int chi[2] = {0, 0}, kap = 0;
  double2* cur = nullptr;
  cudaMemcpyAsync(chi, h->T.lam_chi + B, sizeof(int) * 2, cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(&kap, h->T.site_kappa + s, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(&cur, h->T.site_gam + s, sizeof(double2*), cudaMemcpyDeviceToHost, h->stream);
  int rc = read_status(h);
  if (rc != PT_OK) return rc;
  const size_t n = (size_t)chi[0] * 4 * kap * chi[1];
  if (out) {
    if (cap < n) return h->fail(PT_ERR_ARG, "get_gamma: output holds fewer than chi_l * 4 * kappa * chi_r elements");
    cudaMemcpyAsync(out, cur, sizeof(double2) * n, cudaMemcpyDeviceToHost, h->stream);
    rc = read_status(h);
    if (rc != PT_OK) return rc;
  }
  return (int)n;
}

int pt_tebd_clone(pt_tebd_t h, pt_tebd_t* out) {
  if (!h || !out) return PT_ERR_ARG;
  *out = nullptr;
  int rc = read_status(h);
  if (rc != PT_OK) return rc;
  pt_tebd* c = new pt_tebd();
  c->stream = h->stream;
  c->opt = h->opt;
  c->chains = h->chains;
  c->mpos_in = h->mpos_in;
  rc = build(c);
  if (rc != PT_OK) {
    g_err = c->err;
    c->release();
    delete c;
    return rc;
  }
  // copy the live state: current Gamma buffers, lambdas, dims, log-norms, step, history
  std::vector<double2*> cur(h->n_sites);
  cudaMemcpyAsync(cur.data(), h->T.site_gam, sizeof(double2*) * h->n_sites, cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  for (int s = 0; s < h->n_sites; ++s)
    cudaMemcpyAsync(c->gam_a[s], cur[s], sizeof(double2) * h->site_cap_h[s], cudaMemcpyDeviceToDevice, h->stream);
  for (int B = 0; B < h->n_lams; ++B)
    cudaMemcpyAsync(c->lam_buf[B], h->lam_buf[B], sizeof(double) * h->lam_cap_h[B], cudaMemcpyDeviceToDevice,
                    h->stream);
  cudaMemcpyAsync(c->T.lam_chi, h->T.lam_chi, sizeof(int) * h->n_lams, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(c->T.lam_lognorm, h->T.lam_lognorm, sizeof(double) * h->n_lams, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(c->T.site_kappa, h->T.site_kappa, sizeof(int) * h->n_sites, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(c->T.step, h->T.step, sizeof(int), cudaMemcpyDeviceToDevice, h->stream);
  c->steps_done = h->steps_done;
  cudaStreamSynchronize(h->stream);
  rc = check_cuda(c, "clone");
  if (rc == PT_OK && c->opt.use_graph) rc = capture_graph(c);
  if (rc != PT_OK) {
    c->release();
    delete c;
    return rc;
  }
  *out = c;
  return PT_OK;
}

int pt_tebd_destroy(pt_tebd_t h) {
  if (!h) return PT_ERR_ARG;
  h->release();
  delete h;
  return PT_OK;
}

int pt_tebd_get_svd_sweeps(pt_tebd_t h, int* out, int cap) {
  if (!h || !out || cap < 0) return PT_ERR_ARG;
  const int n = std::min(cap, (int)h->bond_info.size());
  std::vector<int> buf(8);
  for (int i = 0; i < n; ++i) {
    cudaMemcpyAsync(buf.data(), h->bond_info[i], sizeof(int) * 8, cudaMemcpyDeviceToHost, h->stream);
    cudaStreamSynchronize(h->stream);
    out[2 * i] = buf[3];
    out[2 * i + 1] = buf[6];         // the update's fault flags
  }
  int rc = read_status(h);
  return rc == PT_OK ? (int)h->bond_info.size() : rc;
}

int pt_tebd_set_timing(pt_tebd_t h, int enable) {
  if (!h) return PT_ERR_ARG;
  h->timing = enable != 0;
  return PT_OK;
}

int pt_tebd_get_timing(pt_tebd_t h, double* ms9) {
  if (!h || !ms9) return PT_ERR_ARG;
  for (int k = 0; k < 9; ++k) ms9[k] = h->stage_ms[k];
  return PT_OK;
}

// ---------------------------------------------------------------- standalone batched SVD
static size_t svd_layout(int m, int n, int batch, size_t* offs) {
  const int Ma = std::max(m, n), Na = std::min(m, n);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += (bytes + 255) & ~size_t(255);
    return r;
  };
  offs[0] = take(sizeof(double2) * (size_t)Ma * Na * batch);  // A
  offs[1] = take(sizeof(double2) * (size_t)Na * Na * batch);  // V
  offs[2] = take(sizeof(double) * (size_t)Na * batch);        // sig
  offs[3] = take(sizeof(int) * (size_t)Na * batch);           // perm
  offs[4] = take(sizeof(int) * 8 * (size_t)batch);            // info
  offs[5] = take(sizeof(int));                                // status
  offs[6] = take(sizeof(BondWork) * (size_t)batch);           // work items
  offs[7] = take(sizeof(double) * (size_t)Na * batch);        // column norms
  return o;
}

size_t pt_svd_scratch_bytes(int m, int n, int batch) {
  if (m < 1 || n < 1 || batch < 1) return 0;
  size_t offs[8];
  return svd_layout(m, n, batch, offs);
}

static size_t hqr_layout(int m, int n, int batch, size_t* offs) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += (bytes + 255) & ~size_t(255);
    return r;
  };
  offs[0] = take(sizeof(ptk::QRItem) * (size_t)batch);
  offs[1] = take(sizeof(double2) * (size_t)m * n * batch);     // reflectors
  offs[2] = take(sizeof(double) * (size_t)n * batch);          // tau
  offs[3] = take(sizeof(unsigned) * 4);                        // grid barrier
  offs[4] = take(sizeof(int));                                 // status
  return o;
}

size_t pt_qr_scratch_bytes(int m, int n, int batch) {
  if (m < 1 || n < 1 || n > m || batch < 1) return 0;
  size_t offs[5];
  return hqr_layout(m, n, batch, offs);
}

int pt_qr_f64(double* A, int m, int n, int batch, double* R, void* scratch, void* cuda_stream) {
  if (!A || !R || !scratch || m < 1 || n < 1 || n > m || batch < 1 || batch > 2048) {
    g_err = "pt_qr_f64: bad arguments (need 1 <= n <= m, 1 <= batch <= 2048)";
    return PT_ERR_ARG;
  }
  const int blocks = ptk::jacobi_grid_blocks();
  if (blocks <= 0 || !ptk::hqr_items_ok()) {
    g_err = "pt_qr_f64: the device cannot co-schedule the whole-GPU kernel";
    return PT_ERR_CUDA;
  }
  if ((long long)n * batch > (long long)blocks * 384) {
    g_err = "pt_qr_f64: n x batch exceeds the kernel's column capacity";
    return PT_ERR_CAPACITY;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  size_t offs[5];
  hqr_layout(m, n, batch, offs);
  char* base = (char*)scratch;
  ptk::QRItem* items = (ptk::QRItem*)(base + offs[0]);
  unsigned* sync3 = (unsigned*)(base + offs[3]);
  int* status = (int*)(base + offs[4]);
  std::vector<ptk::QRItem> h(batch);
  for (int b = 0; b < batch; ++b)
    h[b] = ptk::QRItem{(double2*)A + (size_t)b * m * n, (double2*)(base + offs[1]) + (size_t)b * m * n,
                       (double2*)R + (size_t)b * n * n, (double*)(base + offs[2]) + (size_t)b * n, m, n};
  cudaMemcpyAsync(items, h.data(), sizeof(ptk::QRItem) * batch, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(status, 0, sizeof(int), st);
  ptk::launch_hqr_items(items, batch, blocks, sync3, status, st);
  int hs = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    g_err = std::string("pt_qr_f64: ") + cudaGetErrorString(e);
    return PT_ERR_CUDA;
  }
  if (hs & ST_TIMEOUT) {
    g_err = "pt_qr_f64: a grid barrier wait ran out of time";
    return PT_ERR_DEVICE_TIMEOUT;
  }
  if (hs & ST_CAPACITY) {
    g_err = "pt_qr_f64: capacity";
    return PT_ERR_CAPACITY;
  }
  return PT_OK;
}

static size_t zgemm_layout(int m, int n, int k, int batch, size_t* offs) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += (bytes + 255) & ~size_t(255);
    return r;
  };
  offs[0] = take(sizeof(ptk::ZGemmItem) * (size_t)batch);
  offs[1] = take(sizeof(int));                                            // status
  offs[2] = take(ptk::zgemm_pack_bytes(m, k, 0) * (size_t)batch);         // packed A
  offs[3] = take(ptk::zgemm_pack_bytes(n, k, 1) * (size_t)batch);         // packed B
  return o;
}

size_t pt_zgemm_scratch_bytes(int m, int n, int k, int batch) {
  if (m < 1 || n < 1 || k < 1 || batch < 1) return 0;
  size_t offs[4];
  return zgemm_layout(m, n, k, batch, offs);
}

int pt_zgemm_sliced(int opA, int opB, int m, int n, int k, const double* A, int lda, long long strideA,
                    const double* B, int ldb, long long strideB, double* C, int ldc, long long strideC, int batch,
                    void* scratch, void* cuda_stream) {
  auto bad = [](const char* why) {
    g_err = std::string("pt_zgemm_sliced: ") + why;
    return PT_ERR_ARG;
  };
  if (m < 1 || n < 1 || k < 1 || batch < 1 || !A || !B || !C || !scratch) return bad("bad arguments");
  if (opA < 0 || opA > 2 || opB < 0 || opB > 2) return bad("op must be 0 (N), 1 (T) or 2 (H)");
  if (lda < (opA == 0 ? m : k) || ldb < (opB == 0 ? k : n) || ldc < m) return bad("leading dimension too small");
  if (batch > 1024) return bad("batch > 1024");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  size_t offs[4];
  zgemm_layout(m, n, k, batch, offs);
  char* base = (char*)scratch;
  ptk::ZGemmItem* items = (ptk::ZGemmItem*)(base + offs[0]);
  int* status = (int*)(base + offs[1]);
  const size_t pa = ptk::zgemm_pack_bytes(m, k, 0), pb = ptk::zgemm_pack_bytes(n, k, 1);
  std::vector<ptk::ZGemmItem> h(batch);
  for (int b = 0; b < batch; ++b) {
    ptk::ZGemmItem it{};
    it.A = (const double2*)A + (size_t)b * strideA;
    it.B = (const double2*)B + (size_t)b * strideB;
    it.C = (double2*)C + (size_t)b * strideC;
    it.lda = lda;
    it.ldb = ldb;
    it.ldc = ldc;
    it.M = m;
    it.N = n;
    it.K = k;
    it.opA = opA;
    it.opB = opB;
    it.TA = (unsigned char*)(base + offs[2]) + (size_t)b * pa;
    it.TB = (unsigned char*)(base + offs[3]) + (size_t)b * pb;
    it.cap_m = m;
    it.cap_n = n;
    it.cap_k = k;
    h[b] = it;
  }
  cudaMemcpyAsync(items, h.data(), sizeof(ptk::ZGemmItem) * batch, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(status, 0, sizeof(int), st);
  ptk::launch_zgemm(items, batch, ptk::zgemm_tile_cap(m, n) * batch, m, n, status, st);
  int hs = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);      // also keeps h alive for the copy above
  if (e != cudaSuccess) {
    g_err = std::string("pt_zgemm_sliced: ") + cudaGetErrorString(e);
    return PT_ERR_CUDA;
  }
  if (hs & ST_TIMEOUT) {
    g_err = "pt_zgemm_sliced: an mbarrier wait ran out of time";
    return PT_ERR_DEVICE_TIMEOUT;
  }
  if (hs & ST_CAPACITY) {
    g_err = "pt_zgemm_sliced: capacity";
    return PT_ERR_CAPACITY;
  }
  return PT_OK;
}

int pt_svd_f64(const double* A, int m, int n, int batch, double* sigma, double* U, double* V,
               void* scratch, int max_sweeps, void* cuda_stream) {
  if (!A || m < 1 || n < 1 || batch < 1 || !sigma || !U || !V || !scratch) {
    g_err = "pt_svd_f64: bad arguments";
    return PT_ERR_ARG;
  }
  if (max_sweeps <= 0) max_sweeps = 60;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  size_t offs[8];
  svd_layout(m, n, batch, offs);
  char* base = (char*)scratch;
  double2* wA = (double2*)(base + offs[0]);
  double2* wV = (double2*)(base + offs[1]);
  double* sig = (double*)(base + offs[2]);
  int* perm = (int*)(base + offs[3]);
  int* info = (int*)(base + offs[4]);
  int* status = (int*)(base + offs[5]);
  BondWork* items = (BondWork*)(base + offs[6]);
  const int Ma = std::max(m, n), Na = std::min(m, n);
  const size_t sA = (size_t)Ma * Na, sV = (size_t)Na * Na;
  std::vector<BondWork> hw(batch);
  std::vector<int> hinfo(8 * (size_t)batch, 0);
  for (int b = 0; b < batch; ++b) {
    BondWork W{};
    W.A = wA + b * sA;
    W.V = wV + b * sV;
    W.sig = sig + (size_t)b * Na;
    W.perm = perm + (size_t)b * Na;
    W.info = info + 8 * (size_t)b;
    W.aux = (double*)(base + offs[7]) + (size_t)b * Na;
    W.mD_cap = m;
    W.nD_cap = n;
    W.k_cap = Na;
    hw[b] = W;
    hinfo[8 * b + 0] = m;
    hinfo[8 * b + 1] = n;
    hinfo[8 * b + 2] = m < n ? 1 : 0;
  }
  cudaMemcpyAsync(items, hw.data(), sizeof(BondWork) * batch, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(info, hinfo.data(), sizeof(int) * hinfo.size(), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(status, 0, sizeof(int), st);
  const int gx = (int)std::min<size_t>(256, ((size_t)m * n + 255) / 256);
  ptk::k_svd_load<<<dim3(gx, batch), 256, 0, st>>>((const double2*)A, m, n, batch, wA, sA);
  const int cl = ptk::jacobi_cluster_size(std::max(1, std::min(16, (Na / 2 + 7) / 8)));
  ptk::launch_jacobi_cluster(items, batch, cl, max_sweeps, status, st);
  const int gs = (int)std::min<size_t>(256, ((size_t)(m + n + 1) * Na + 255) / 256);
  ptk::k_svd_store<<<dim3(gs, batch), 256, 0, st>>>(wA, wV, sig, perm, m, n, batch, sA, sV, sigma,
                                                    (double2*)U, (double2*)V);
  // the host copies of items/info must outlive the async copies above
  cudaError_t es = cudaStreamSynchronize(st);
  if (es != cudaSuccess) {
    g_err = std::string("pt_svd_f64: ") + cudaGetErrorString(es);
    return PT_ERR_CUDA;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_err = std::string("pt_svd_f64: ") + cudaGetErrorString(e);
    return PT_ERR_CUDA;
  }
  int hs = 0;
  e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    g_err = std::string("pt_svd_f64: ") + cudaGetErrorString(e);
    return PT_ERR_CUDA;
  }
  if (hs & ST_SVD_NOCONV) {
    g_err = "pt_svd_f64: Jacobi did not converge";
    return PT_ERR_SVD_NOCONV;
  }
  if (hs & ST_NAN) {
    g_err = "pt_svd_f64: NaN";
    return PT_ERR_NAN;
  }
  return PT_OK;
}

}  // extern "C"
