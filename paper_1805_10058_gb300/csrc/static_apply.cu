// Allocation-free 3D operator apply (cd_apply3d_static): bands, per-RHS parameters and the
// work arrays of the three banded passes live in one fixed-size file-scope device array, so
// the call never allocates device memory.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "cd_internal.h"

namespace cd {

// 48 MiB, reserved on every device that loads this library, for as long as it stays loaded.
static constexpr size_t kStaticScratchBytes = size_t(48) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void* g_static_dev_ptr[128] = {};  // device address of g_static_scratch, per device

// True while `p` is still device memory of device `dev` (a cached address goes stale when the
// process resets the device and its context is rebuilt).
static bool still_device_ptr(void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Device address of the array on the current device; looked up once per device (and again if
// the device's context was rebuilt since).
static cd_status static_scratch_ptr(void** out) {
  int dev = 0;
  CD_CUDA_OK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) {
    set_error("cd_apply3d_static: device ordinal out of range");
    return CD_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (g_static_dev_ptr[dev] && !still_device_ptr(g_static_dev_ptr[dev], dev))
    g_static_dev_ptr[dev] = nullptr;
  if (!g_static_dev_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cd_apply3d_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return CD_ECUDA;
    }
    g_static_dev_ptr[dev] = p;
  }
  *out = g_static_dev_ptr[dev];
  return CD_OK;
}

}  // namespace cd

extern "C" cd_status cd_apply3d_static(int p, int n, double alpha, double beta, const double* w,
                                       double* y, int nrhs, void* cuda_stream) {
  using namespace cd;
  if (!w || !y || nrhs < 1 || p < 1 || n < 1 || n + p - 2 < 2) {
    set_error("cd_apply3d_static: need w, y != NULL, nrhs >= 1, p >= 1, n >= 1, n + p - 2 >= 2");
    return CD_EINVAL;
  }
  if (!(alpha > 0) || !(beta > 0) || !std::isfinite(alpha) || !std::isfinite(beta)) {
    set_error("cd_apply3d_static: alpha and beta must be finite and > 0");
    return CD_EINVAL;
  }
  const int m = n + p - 2, P = p, W = 2 * P + 1;
  // layout (doubles): bands [3][m][W] | alpha[nrhs] | beta[nrhs] | 18 arrays of m^3 nrhs (the
  // two groups of nine intermediates of the three banded FP64 passes, which write y directly)
  const size_t n3 = (size_t)m * m * m;
  const size_t nb = ((size_t)3 * m * W + 31) / 32 * 32;
  const size_t np = ((size_t)2 * nrhs + 31) / 32 * 32;
  const size_t need = nb + np + (size_t)18 * n3 * nrhs;
  if (need * sizeof(double) > kStaticScratchBytes) {
    set_error("cd_apply3d_static: (m, nrhs) too large for the 48 MiB static scratch (it needs about "
              "18 m^3 nrhs + 3 m (2p+1) + 2 nrhs doubles; m = " + std::to_string(m) +
              ", nrhs = " + std::to_string(nrhs) + ")");
    return CD_EINVAL;
  }
  void* base = nullptr;
  cd_status st = static_scratch_ptr(&base);
  if (st != CD_OK) return st;
  double* dbands = static_cast<double*>(base);
  double* dal = dbands + nb;
  double* dbe = dal + nrhs;
  double* dscr = dbands + nb + np;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  Band M, A, S;
  iga_bands(p, n, P, M, A, S);
  std::vector<double> host(nb + 2 * (size_t)nrhs, 0.0);
  std::copy(M.v.begin(), M.v.end(), host.begin());
  std::copy(A.v.begin(), A.v.end(), host.begin() + (size_t)m * W);
  std::copy(S.v.begin(), S.v.end(), host.begin() + (size_t)2 * m * W);
  for (int i = 0; i < nrhs; ++i) {
    host[nb + i] = alpha;
    host[nb + nrhs + i] = beta;
  }
  // every region the kernels read is rewritten here or by an earlier pass of this call.  The
  // source is pageable host memory: CUDA stages it before cudaMemcpyAsync returns, so the
  // vector may go out of scope without waiting for the copy.
  CD_CUDA_OK(cudaMemcpyAsync(dbands, host.data(), host.size() * sizeof(double),
                             cudaMemcpyHostToDevice, s));
  if (launch_apply<double>(3, m, P, dbands, w, y, nullptr, 0, nrhs, Coef{dal, dbe}, nullptr,
                           nullptr, nullptr, dscr, s) != 0) {
    set_error("cd_apply3d_static: no apply kernel fits this problem size");
    return CD_EINVAL;
  }
  CD_CUDA_OK(cudaGetLastError());
  return CD_OK;
}
