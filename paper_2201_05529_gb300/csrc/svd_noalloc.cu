// pt_svd_f64_noalloc: the batched FP64 Jacobi SVD entry point for callers that cannot allocate
// device memory.
//
// Some callers own every byte of device memory through their own pool (a framework that reserves
// the GPU up front, a fixed-budget service) or run where a device allocation is not acceptable
// (cudaMalloc may synchronise the whole device and can fail under memory pressure in the middle
// of a job). They cannot provide the workspace that pt_svd_f64 asks for. This entry point instead
// uses one file-scope device array of fixed size as its workspace; the caller passes only inputs
// and outputs.
//
// Properties a caller must know:
//  * The workspace is a static __device__ array of PT_SVD_NOALLOC_MAX_BYTES bytes. Every GPU that
//    loads this library holds it until the process exits.
//  * Problems whose workspace would exceed that size are rejected with PT_ERR_CAPACITY.
//  * The first call on a device looks up the array's device address (cudaGetSymbolAddress, with
//    that device current) and caches it per device index. A cudaDeviceReset invalidates that
//    cached address: after a reset, reload the library before calling again.
//  * Every call reads the device status word back and synchronises its stream before returning,
//    so no call (the first or a later one) may be made while that stream is being captured.
//  * Every call shares the one array. Calls that overlap on the GPU (different streams, or host
//    threads without ordering) race on it and corrupt each other's results; serialise them.
//  * The array keeps the previous call's contents; everything that must start at zero is cleared
//    by the call itself (status word, convergence counters, V, work descriptors).
// No cudaMalloc, cudaFree or other allocating routine is called on this path.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>

#include "kernels.h"
#include "../../include/pt_tebd.h"

namespace {

constexpr size_t NOALLOC_BYTES = PT_SVD_NOALLOC_MAX_BYTES;
static __device__ __align__(256) unsigned char g_svd_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mu;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t A, V, sig, perm, info, status, items, aux, total;
};

Layout layout(int m, int n, int batch) {
  const size_t Ma = m > n ? m : n, Na = m < n ? m : n;
  Layout L;
  size_t o = 0;
  L.A = o; o += align256(sizeof(double2) * Ma * Na * batch);
  L.V = o; o += align256(sizeof(double2) * Na * Na * batch);
  L.sig = o; o += align256(sizeof(double) * Na * batch);
  L.perm = o; o += align256(sizeof(int) * Na * batch);
  L.info = o; o += align256(sizeof(int) * 8 * (size_t)batch);
  L.status = o; o += align256(sizeof(int));
  L.items = o; o += align256(sizeof(BondWork) * (size_t)batch);
  L.aux = o; o += align256(sizeof(double) * Na * batch);
  L.total = o;
  return L;
}

// Fill the per-matrix work descriptors in the workspace on the device (no host staging buffers).
__global__ void k_noalloc_setup(unsigned char* base, Layout L, int m, int n, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) *(int*)(base + L.status) = 0;
  if (b >= batch) return;
  const size_t Ma = m > n ? m : n, Na = m < n ? m : n;
  BondWork W{};
  W.A = (double2*)(base + L.A) + b * Ma * Na;
  W.V = (double2*)(base + L.V) + b * Na * Na;
  W.sig = (double*)(base + L.sig) + b * Na;
  W.aux = (double*)(base + L.aux) + b * Na;
  W.perm = (int*)(base + L.perm) + b * Na;
  W.info = (int*)(base + L.info) + 8 * b;
  W.mD_cap = m;
  W.nD_cap = n;
  W.k_cap = (int)Na;
  for (int i = 0; i < 8; ++i) W.info[i] = 0;
  W.info[0] = m;
  W.info[1] = n;
  W.info[2] = m < n ? 1 : 0;
  ((BondWork*)(base + L.items))[b] = W;
}

int fail(int code, const std::string& msg) {
  ptk::set_global_error(("pt_svd_f64_noalloc: " + msg).c_str());   // read with pt_tebd_last_error(NULL)
  return code;
}

// Device address of the static workspace for the current device (looked up once per device).
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= MAX_DEVICES) return fail(PT_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_svd_scratch);
    if (e != cudaSuccess || !p)
      return fail(PT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return PT_OK;
}

}  // namespace

extern "C" {

int pt_svd_f64_noalloc(const double* A, int m, int n, int batch, double* sigma, double* U, double* V,
                       int max_sweeps, void* cuda_stream) {
  if (!A || m < 1 || n < 1 || batch < 1 || !sigma || !U || !V) return fail(PT_ERR_ARG, "bad arguments");
  const Layout L = layout(m, n, batch);
  if (L.total > NOALLOC_BYTES)
    return fail(PT_ERR_CAPACITY, "problem needs " + std::to_string(L.total) + " bytes of workspace, more than the " +
                                     std::to_string(NOALLOC_BYTES) + "-byte static array");
  if (max_sweeps <= 0) max_sweeps = 60;
  void* addr = nullptr;
  int rc = scratch_address(&addr);
  if (rc != PT_OK) return rc;
  unsigned char* base = (unsigned char*)addr;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int Ma = m > n ? m : n, Na = m < n ? m : n;
  const size_t sA = (size_t)Ma * Na, sV = (size_t)Na * Na;
  k_noalloc_setup<<<(batch + 127) / 128, 128, 0, st>>>(base, L, m, n, batch);
  const int gx = (int)std::min<size_t>(256, ((size_t)m * n + 255) / 256);
  ptk::k_svd_load<<<dim3(gx, batch), 256, 0, st>>>((const double2*)A, m, n, batch, (double2*)(base + L.A), sA);
  const int cl = ptk::jacobi_cluster_size(std::max(1, std::min(16, (Na / 2 + 7) / 8)));
  ptk::launch_jacobi_cluster((const BondWork*)(base + L.items), batch, cl, max_sweeps,
                             (int*)(base + L.status), st);
  const int gs = (int)std::min<size_t>(256, ((size_t)(m + n + 1) * Na + 255) / 256);
  ptk::k_svd_store<<<dim3(gs, batch), 256, 0, st>>>((const double2*)(base + L.A), (const double2*)(base + L.V),
                                                    (const double*)(base + L.sig), (const int*)(base + L.perm), m,
                                                    n, batch, sA, sV, sigma, (double2*)U, (double2*)V);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PT_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  int hs = 0;
  e = cudaMemcpyAsync(&hs, base + L.status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(PT_ERR_CUDA, std::string("sync: ") + cudaGetErrorString(e));
  if (hs & ST_SVD_NOCONV) return fail(PT_ERR_SVD_NOCONV, "Jacobi did not converge within max_sweeps");
  if (hs & ST_NAN) return fail(PT_ERR_NAN, "NaN in the singular values");
  return PT_OK;
}

}  // extern "C"
