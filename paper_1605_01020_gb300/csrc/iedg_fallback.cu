// FP64 fallback of the mixed-precision forms: elements whose FP32 / low-precision
// condensation did not give FP64-accurate results are condensed again in FP64 in the
// same call, with the FP64 kernels of the FP64 path.
//
// An element qualifies when its refinement did not reach the tolerance
// (IEDG_ELEM_REFINE), when a tensor-core completion wait gave up on it
// (IEDG_ELEM_TIMEOUT), or when its FP32 partial LU met an exact zero pivot
// (IEDG_ELEM_SINGULAR; rounding can make a pivot vanish in FP32 only).  Up to
// kFallbackSlots of them, lowest element ids first, get a slot: the FP64 bordered
// matrix is assembled into the slot from the FP64 point Jacobians and lifted operators
// the mixed path keeps anyway, factored by the FP64 partial LU, and then
//   K_e      is read from the slot by the BSR gather (scatter_K),
//   R_e      is copied from the slot into the element's FP64 trace residual,
//   dZ_e     comes from the slot's factors in the back-substitution.
// A recomputed element reports IEDG_ELEM_FALLBACK (or the FP64 LU's own status);
// qualifying elements past the slots keep their flag.  Everything runs on the device
// with fixed grids (no host synchronisation): the slot list is built by one CTA and
// the other kernels skip empty slots.
#include "iedg_internal.cuh"

namespace iedg {
namespace {

constexpr int FB_SELECT_THREADS = 1024;

__device__ __forceinline__ bool fb_qualifies(int8_t s) {
  return s == IEDG_ELEM_REFINE || s == IEDG_ELEM_TIMEOUT || s == IEDG_ELEM_SINGULAR;
}

// slot_of[e] = slot of element e or -1; list[slot] = element or -1; *count = slots used.
__global__ void __launch_bounds__(FB_SELECT_THREADS)
k_fb_select(const int8_t* __restrict__ status, int64_t E, int n_slots, int64_t* __restrict__ list,
            int* __restrict__ slot_of, int* __restrict__ count) {
  __shared__ int part[FB_SELECT_THREADS];
  const int tid = threadIdx.x;
  const int64_t chunk = (E + FB_SELECT_THREADS - 1) / FB_SELECT_THREADS;
  const int64_t lo = tid * chunk, hi = min(E, lo + chunk);
  int c = 0;
  for (int64_t e = lo; e < hi; ++e) c += fb_qualifies(status[e]);
  part[tid] = c;
  __syncthreads();
  // exclusive scan of the per-thread counts (Hillis-Steele on the shared array)
  for (int o = 1; o < FB_SELECT_THREADS; o <<= 1) {
    const int v = tid >= o ? part[tid - o] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int k = part[tid] - c;
  for (int64_t e = lo; e < hi; ++e) {
    int sl = -1;
    if (fb_qualifies(status[e])) {
      if (k < n_slots) { sl = k; list[k] = e; }
      ++k;
    }
    slot_of[e] = sl;
  }
  const int total = part[FB_SELECT_THREADS - 1];
  for (int s = tid; s < n_slots; s += FB_SELECT_THREADS)
    if (s >= total) list[s] = -1;
  if (tid == 0) *count = min(total, n_slots);
}

// Status and trace residual of the recomputed elements: R_e = the slot's trace rows of
// the right-hand-side column (component-major, as the refinement writes it).
__global__ void k_fb_finish(Dims dm, const int64_t* __restrict__ list, const int8_t* __restrict__ fb_status,
                            const double* __restrict__ S, double* __restrict__ re64, int8_t* __restrict__ status) {
  const int64_t slot = blockIdx.x;
  const int64_t e = list[slot];
  if (e < 0) return;
  const double* A = S + slot * (int64_t)dm.n * dm.ld;
  for (int r = threadIdx.x; r < dm.nt; r += blockDim.x) re64[e * dm.nt + r] = A[(int64_t)(dm.nu + r) * dm.ld + dm.n];
  if (threadIdx.x == 0) status[e] = fb_status[slot] == IEDG_ELEM_OK ? IEDG_ELEM_FALLBACK : fb_status[slot];
}

}  // namespace

cudaError_t launch_fallback(iedg_mesh* M, cudaStream_t st) {
  if (M->fb_S == nullptr) return cudaSuccess;
  const int ns = kFallbackSlots;
  k_fb_select<<<1, FB_SELECT_THREADS, 0, st>>>(M->status, M->E, ns, M->fb_list, M->fb_slot, M->fb_count);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = launch_assemble_list(M, M->fb_S, M->fb_list, ns, st);
  if (err == cudaSuccess && M->fault.zero_row_elem >= 0) err = launch_zero_row_fallback(M, st);
  if (err == cudaSuccess) err = launch_lu64_list(M, M->fb_S, ns, M->fb_list, M->fb_status, st);
  if (err != cudaSuccess) return err;
  k_fb_finish<<<ns, 128, 0, st>>>(M->dm, M->fb_list, M->fb_status, M->fb_S, M->re64, M->status);
  return cudaGetLastError();
}

}  // namespace iedg
