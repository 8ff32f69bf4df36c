// Pieces shared by the batched partial-LU kernels (FP64, FP32 and tensor-core forms):
// element descriptors, the persistent element queue, the tensor-core state of a CTA
// and the grid of the persistent launch.
#pragma once
#include "iedg_internal.cuh"
#include "iedg_tc.cuh"

namespace iedg {
namespace {

constexpr int LU_THREADS = 256;
constexpr int UCW = 64;     // trailing-update column chunk
constexpr int LU_MAX_NU = 640;   // u-unknowns of the largest element (5 x 125 at p = 4)

// Tensor-core state of a CTA (deferred Schur complement forms of the LU).
struct TcState {
  uint32_t tmem;        // TMEM base
  uint64_t* mbar;       // MMA completion barriers (one per operand stage)
  uint32_t phase[2];    // parity of each barrier's next completion
  int failed;           // a completion wait ran out
  int limit;            // polls of a completion wait before it gives up (0: gives up at once)
  int pending[2];       // a commit on barrier b has not been waited for yet
};

// Drain after a failed wait: the MMAs still in flight complete (bounded, full limit)
// before the CTA frees its TMEM; barriers with no commit outstanding are skipped.
__device__ __forceinline__ void tc_drain(const TcState& t) {
  for (int b = 0; b < 2; ++b)
    if (t.pending[b]) tc::mbar_wait(t.mbar + b, t.phase[b], kTcWaitLimit);
}

// Sizes and location of one element's bordered matrix.
struct LuElem {
  int n, nu, ld;
  int64_t off, poff;
};

__device__ __forceinline__ LuElem lu_elem(const Dims& dm, const LuDesc& lud, int64_t e) {
  if (lud.soff) return LuElem{lud.n[e], lud.nu[e], lud.ld[e], lud.soff[e], lud.poff ? lud.poff[e] : 0};
  return LuElem{dm.n, dm.nu, dm.ld, e * (int64_t)dm.n * dm.ld, e * (int64_t)dm.nu};
}

// Element scheduling of the batched LU.  queue == nullptr: one CTA per element.
// Otherwise a persistent grid (a few CTAs per SM) takes elements from an atomic
// counter in order, so no SM idles in a partial last wave.
// With an order list the k-th element taken is order[k].
__device__ __forceinline__ bool next_element(int64_t* queue, int64_t E, int64_t it, const int64_t* order,
                                             int64_t* e_out) {
  __shared__ unsigned long long s_next;
  if (queue == nullptr) {
    *e_out = order ? order[blockIdx.x] : (int64_t)blockIdx.x;
    return it == 0;
  }
  if (threadIdx.x == 0) s_next = atomicAdd(reinterpret_cast<unsigned long long*>(queue), 1ull);
  __syncthreads();
  const int64_t k = (int64_t)s_next;
  __syncthreads();
  *e_out = (order && k < E) ? order[k] : k;
  return k < E;
}

}  // namespace

// Grid of the persistent form: resident CTAs per SM x SMs (never more than E).  The
// kernel asks for the largest shared-memory carveout first, so the occupancy query
// sees the split the launch will get.
template <class K>
static inline cudaError_t persistent_grid(K kern, size_t smem, int64_t E, unsigned* grid, int max_per_sm = 64,
                                          int threads = LU_THREADS) {
  int dev = 0, sms = 0, per_sm = 0, smem_sm = 0, reserved = 0;
  cudaFuncAttributes fa;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
  if (err == cudaSuccess) err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (err == cudaSuccess) err = cudaFuncGetAttributes(&fa, kern);
  if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (err != cudaSuccess) return err;
  // the same bound from the kernel's own shared memory, registers and threads (the
  // occupancy query has been seen to answer one block less than fits for the largest
  // shared-memory configurations); a grid above what fits only queues blocks
  int own = smem_sm / (int)(smem + fa.sharedSizeBytes + reserved);
  if (fa.numRegs > 0) own = own < 65536 / (fa.numRegs * threads) ? own : 65536 / (fa.numRegs * threads);
  own = own < 2048 / threads ? own : 2048 / threads;
  if (own > per_sm) per_sm = own;
  if (per_sm > max_per_sm) per_sm = max_per_sm;
  int64_t g = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  *grid = (unsigned)(g < E ? g : E);
  return cudaSuccess;
}

}  // namespace iedg
