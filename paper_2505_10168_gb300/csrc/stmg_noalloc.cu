// stmg_noalloc.cu -- stmg_sensitivity_noalloc: the design sensitivity without any
// device allocation.
//
// stmg_sensitivity needs a handle (whose creation allocates the level hierarchy) and
// per-call scratch for the partial sums over time chunks.  Some callers cannot allocate
// device memory at the point where they need a gradient: cudaMalloc and cudaFree can
// synchronise the whole device, which a caller that keeps other streams busy (an
// optimisation loop overlapping its own kernels with ours) cannot afford, and callers
// whose device memory is fixed at start-up by a framework-owned pool or a hard memory
// budget are not allowed to request more.  This variant takes every input and output
// from the caller and keeps its scratch in a fixed-size array in the library's device
// image, which every GPU that loads the library holds until the process exits.
#include <cstdio>
#include <mutex>

#include "stmg.h"
#include "stmg_internal.h"
#include "stmg_placement.h"

namespace stmg {
namespace {

// Partial sums of the sensitivity, two values per (time chunk, element).
__device__ __align__(256) double g_noalloc_scratch[STMG_NOALLOC_MAX_SCRATCH];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per device;
// host code only sees a stand-in for the symbol, never its device address).
stmg_status scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_global_error("stmg_sensitivity_noalloc: no usable current device");
    return STMG_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      char buf[256];
      snprintf(buf, sizeof buf, "stmg_sensitivity_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      set_global_error(buf);
      return STMG_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return STMG_OK;
}

// Where a pointer lives relative to the current device (kPlaceUsable, kPlaceOtherDevice
// or kPlaceNotDevice; an unknown pointer counts as host memory).
int placement(const void* p, int current_device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return kPlaceNotDevice;
  }
  return noalloc_placement(static_cast<int>(a.type), a.device, current_device);
}

}  // namespace
}  // namespace stmg

using namespace stmg;

extern "C" stmg_status stmg_sensitivity_noalloc(int nel, int nt, double L, double t_end, const double* chi,
                                                const double* simp6, const double* u, const double* lam,
                                                double* dtheta_dchi, void* stream) {
  if (nel < 1 || nt < 1 || nt > (1 << 30) || !(L > 0.0) || !(t_end > 0.0) || !chi || !simp6 || !u || !lam || !dtheta_dchi) {
    set_global_error("stmg_sensitivity_noalloc: need nel >= 1, 1 <= nt <= 2^30, L > 0, t_end > 0 and non-NULL arrays");
    return STMG_EINVAL;
  }
  const long long need = 2LL * sens_chunks(nt) * nel;
  if (need > STMG_NOALLOC_MAX_SCRATCH) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "stmg_sensitivity_noalloc: nel=%d, nt=%d needs %lld scratch values, more than the fixed maximum %d",
             nel, nt, need, STMG_NOALLOC_MAX_SCRATCH);
    set_global_error(buf);
    return STMG_EINVAL;
  }
  if (sens_chunks(nt) > kMaxGridY) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "stmg_sensitivity_noalloc: nt=%d gives %d time chunks of %d rows, more than the %d a launch can hold",
             nt, sens_chunks(nt), kSensRowsPerChunk, kMaxGridY);
    set_global_error(buf);
    return STMG_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    set_global_error("stmg_sensitivity_noalloc: no usable current device");
    return STMG_ECUDA;
  }
  const void* arrays[4] = {chi, u, lam, dtheta_dchi};
  for (const void* a : arrays) {
    const int where = placement(a, dev);
    if (where == kPlaceOtherDevice) {
      set_global_error("stmg_sensitivity_noalloc: chi, u, lam and dtheta_dchi must be on the current device, "
                       "not on another GPU");
      return STMG_EINVAL;
    }
    if (where != kPlaceUsable) {
      set_global_error("stmg_sensitivity_noalloc: chi, u, lam and dtheta_dchi must be device memory");
      return STMG_EINVAL;
    }
  }
  double* scratch = nullptr;
  stmg_status st = scratch_address(&scratch);
  if (st != STMG_OK) return st;
  Simp6 sp;
  for (int i = 0; i < 6; ++i) sp.v[i] = simp6[i];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // u and lam are read in place: their dense rows of nel+1 values are the pitch.  Every
  // scratch slot the reduction reads is written first in the same call, so nothing has
  // to be cleared between calls.
  cudaError_t e = launch_sensitivity(nel, nt, nel + 1, L / nel, t_end / nt, chi, sp, u, lam, scratch, dtheta_dchi, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof buf, "stmg_sensitivity_noalloc: %s", cudaGetErrorString(e));
    set_global_error(buf);
    return STMG_ECUDA;
  }
  return STMG_OK;
}
