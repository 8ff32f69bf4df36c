// Residual entry point that performs no device allocation of its own.
//
// Some callers cannot call cudaMalloc (or anything that allocates) at the point
// where they need a residual: code running while a framework owns the device
// memory pool and must see every allocation, hard real-time loops in which an
// allocation (and the implicit device synchronisation cudaMalloc/cudaFree may
// perform) is not allowed, or plug-ins that are handed device buffers but no
// allocation rights.  iedg_eval_residual_static serves them: apart from the
// caller's inputs and outputs (and the mesh handle created beforehand) it only
// uses the file-scope scratch array below, which every GPU that loads this
// library holds for the lifetime of the process.
#include <mutex>

#include "iedg_internal.cuh"

using namespace iedg;

// Per-element trace residuals R^_e [E][Nb][m] live here instead of in the handle.
static __device__ __align__(256) double g_static_rhat[IEDG_STATIC_SCRATCH_DOUBLES];

namespace {

constexpr int kMaxDevices = 64;
double* g_static_ptr[kMaxDevices] = {nullptr};
std::mutex g_static_mu;

}  // namespace

extern "C" int iedg_eval_residual_static(iedg_mesh* M, const double* u, const double* uhat,
                                         const double* q, const double* u_ref, double* r_u,
                                         double* r_fl, void* stream) {
  if (!M || !u || !uhat || !q || !r_fl) {
    if (M) M->err = "iedg_eval_residual_static: u, uhat, q and r_fl are required";
    return IEDG_ERR_INVALID_ARG;
  }
  if (M->mixed_orders) {
    M->err = "iedg_eval_residual_static: meshes with mixed orders are not supported; use iedg_eval_residual";
    return IEDG_ERR_UNSUPPORTED;
  }
  const Dims& dm = M->dm;
  const int64_t need = M->E * (int64_t)dm.Nb * dm.m;
  if (need > (int64_t)IEDG_STATIC_SCRATCH_DOUBLES) {
    M->err = "iedg_eval_residual_static: mesh needs " + std::to_string(need) +
             " scratch doubles (n_elem * Nb * m), above the static limit of " +
             std::to_string((long long)IEDG_STATIC_SCRATCH_DOUBLES) + "; use iedg_eval_residual";
    return IEDG_ERR_INVALID_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    M->err = std::string("iedg_eval_residual_static: cudaGetDevice: ") + cudaGetErrorString(e);
    return IEDG_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    M->err = "iedg_eval_residual_static: device index " + std::to_string(dev) + " above the " +
             std::to_string(kMaxDevices) + " devices supported by the static entry point";
    return IEDG_ERR_CUDA;
  }
  double* scratch = nullptr;
  {
    // one-time set-up per device, with that device current: the host-side name of
    // g_static_rhat is not a device address, so ask the runtime for it
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
      double* p = nullptr;
      e = cudaGetSymbolAddress((void**)&p, g_static_rhat);
      if (e != cudaSuccess) {
        M->err = std::string("iedg_eval_residual_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return IEDG_ERR_CUDA;
      }
      g_static_ptr[dev] = p;
    }
    scratch = g_static_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  // The point kernel writes every (element, slot, component) entry of the scratch
  // before the gather reads it, so nothing has to be cleared between calls.
  e = launch_points(M, u, q, nullptr, uhat, u_ref, false, r_u, scratch, st);
  if (e == cudaSuccess)
    e = launch_scatter_R(M, scratch, (int64_t)dm.Nb * dm.m, dm.m, 1, r_fl, st);
  if (e != cudaSuccess) {
    M->err = std::string("iedg_eval_residual_static: ") + cudaGetErrorString(e);
    return IEDG_ERR_CUDA;
  }
  return IEDG_OK;
}
