// sv_norm_noalloc: the norm reduction with its partial sums in a static device array instead of memory the
// library allocates, for callers that cannot let the library call cudaMalloc (see include/sv.h).
#include <cstdint>
#include <mutex>
#include <string>
#include <cuda_runtime.h>

#include "sv_internal.h"
#include "../../include/sv.h"

namespace svi {
int set_error(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
int check_device();
} // namespace svi

namespace {

// One slot per block of the first reduction stage.  In host code this name is only a stand-in for the
// device symbol; kernels get its device address from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_norm_partials[SV_NORM_NOALLOC_MAX_PARTIALS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_partials_ptr[kMaxDevices] = {};

// Device address of g_norm_partials on the current device, looked up once per device.
int scratch_for_current_device(double **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return svi::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return svi::set_error(SV_ERR_ARG, "device index beyond the library's table");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_partials_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_norm_partials);
    if (e != cudaSuccess || p == nullptr) return svi::cuda_fail(e, "cudaGetSymbolAddress of the norm scratch");
    g_partials_ptr[dev] = (double *)p;
  }
  *out = g_partials_ptr[dev];
  return SV_OK;
}

} // namespace

extern "C" sv_status sv_norm_noalloc(const void *psi, int n, sv_dtype dtype, void *stream, double *d_out) {
  using namespace svi;
  if (!psi || !d_out) return set_error(SV_ERR_ARG, "psi and d_out must be device pointers, not NULL");
  if (((uintptr_t)psi & 15u) != 0) return set_error(SV_ERR_ARG, "psi must be 16-byte aligned");
  if (((uintptr_t)d_out & 7u) != 0) return set_error(SV_ERR_ARG, "d_out must be 8-byte aligned");
  if (n < 1 || n > kMaxQubits) return set_error(SV_ERR_ARG, "n must be in [1, 36]");
  if (dtype != SV_C64 && dtype != SV_C128) return set_error(SV_ERR_ARG, "dtype must be SV_C64 or SV_C128");
  int rc = check_device();
  if (rc != SV_OK) return rc;
  // Partial count from the SM count of the device current now (the caller may switch devices between calls).
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device attributes");
  const int parts = norm_parts_for_sms(sms);
  if (parts > SV_NORM_NOALLOC_MAX_PARTIALS)
    return set_error(SV_ERR_ARG, "this GPU needs " + std::to_string(parts) + " partial sums; the fixed scratch holds " +
                                     std::to_string(SV_NORM_NOALLOC_MAX_PARTIALS));
  double *partials = nullptr;
  if ((rc = scratch_for_current_device(&partials)) != SV_OK) return rc;
  const int mode = dtype == SV_C64 ? MODE_C64_F32 : MODE_C128_DF32;
  e = launch_norm_parts(psi, n, mode, partials, d_out, (cudaStream_t)stream, 0, parts);
  return e == cudaSuccess ? SV_OK : cuda_fail(e, "norm launch");
}
