// Diagnostic: the bounded grid barrier's failure path, exercised without a GPU fault.
//
// Every spin-wait of the path's cooperative kernels (the Jacobi rounds, the pivoted-QR steps) has
// a time limit after which the waiting CTA records ST_TIMEOUT, raises the launch's abort flag and
// returns, so that a lost CTA surfaces as PT_ERR_DEVICE_TIMEOUT on the host with the context still
// usable. pt_selftest_grid_barrier runs that same barrier code in a small cooperative launch
// (one CTA per SM, three barriers) in which one CTA can be withheld: it returns at once and never
// arrives, so the others wait for the given limit, then time out and leave. The barrier words and
// the status live in static device variables (no allocation); the call synchronises the device.
#include "pt_tebd.h"
#include "grid_sync.cuh"
#include "kernels.h"

namespace ptk {

static __device__ unsigned g_selftest_sync[4];
static __device__ int g_selftest_status;

__global__ void k_barrier_selftest(GridSync gs, int* status, int withheld) {
  if ((int)blockIdx.x == withheld) return;          // this CTA never arrives
  for (int k = 0; k < 3; ++k)
    if (!grid_barrier(gs, status)) return;
}

}  // namespace ptk

extern "C" int pt_selftest_grid_barrier(int withheld_block, double limit_ms, int* device_status) {
  using namespace ptk;
  if (limit_ms <= 0.0 || limit_ms > 10000.0) return PT_ERR_ARG;
  int dev = 0, sms = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PT_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  if (sms <= 0 || khz <= 0) return PT_ERR_CUDA;
  if (withheld_block >= sms) return PT_ERR_ARG;
  unsigned* sync = nullptr;
  int* status = nullptr;
  if (cudaGetSymbolAddress((void**)&sync, g_selftest_sync) != cudaSuccess ||
      cudaGetSymbolAddress((void**)&status, g_selftest_status) != cudaSuccess)
    return PT_ERR_CUDA;
  if (cudaMemset(sync, 0, sizeof(unsigned) * 4) != cudaSuccess || cudaMemset(status, 0, sizeof(int)) != cudaSuccess)
    return PT_ERR_CUDA;
  GridSync gs{sync, (int*)(sync + 2), (long long)(limit_ms * (double)khz)};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sms, 1, 1);
  cfg.blockDim = dim3(32, 1, 1);
  cfg.stream = 0;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_barrier_selftest, gs, status, withheld_block) != cudaSuccess) return PT_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return PT_ERR_CUDA;
  int st = 0;
  if (cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PT_ERR_CUDA;
  if (device_status) *device_status = st;
  return (st & ST_TIMEOUT) ? PT_ERR_DEVICE_TIMEOUT : PT_OK;
}
