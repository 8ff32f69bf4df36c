// Peak-throughput probes of the arithmetic units the element-local path uses, for the
// denominators of its roofline fractions (no counterpart in the paper):
//   FP64 FMA (DFMA), FP32 FMA (FFMA), FP64 tensor MMA (mma.sync m8n8k4 f64, "DMMA"),
//   5th-generation tensor-core MMA (tcgen05.mma) with TF32 and with BF16 operands.
// Each probe keeps its unit busy with independent work from every SM for a fixed
// count of operations and reports FLOP/s from CUDA events around the launch.  Values
// are meaningless (constants); only the timing is used.
//
// C ABI: iedg_peak_probe(kind, reps, &tflops) runs one probe on the current device;
// kind 0 DFMA, 1 FFMA, 2 DMMA, 3 tcgen05 kind::tf32, 4 tcgen05 kind::f16 (BF16).
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;     // independent accumulators per thread

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma(T* out, int iters, T a, T b) {
  T acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  if (s == (T)-1.2345) out[0] = s;     // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(kThreads) k_dmma(double* out, int iters) {
  double acc[kChains][2];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c][0] = acc[c][1] = 0.0;
  const double a = 1.0 + 1e-9 * threadIdx.x, b = 1.0 - 1e-9 * threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(acc[c][0]), "+d"(acc[c][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c][0] + acc[c][1];
  if (s == -1.2345) out[0] = s;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// M = 128, N = 256 (largest single-CTA shape), K-major operands without swizzle:
// A 128 x 32 bytes of K, B 256 x 32 bytes of K, one instruction per K step.
constexpr int kTcM = 128, kTcN = 256;

template <int KIND>   // 0 = kind::tf32 (K = 8), 1 = kind::f16 with BF16 operands (K = 16)
__global__ void __launch_bounds__(128, 1) k_tcgen05(int iters, int* failed) {
  __shared__ __align__(1024) unsigned char a[kTcM * 32];
  __shared__ __align__(1024) unsigned char b[kTcN * 32];
  __shared__ uint32_t tmem;
  __shared__ __align__(8) uint64_t mbar;
  const int tid = threadIdx.x;
  for (int i = tid; i < kTcM * 32 / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(a)[i] = 0x3F800000u ^ (i & 0xFF);
  for (int i = tid; i < kTcN * 32 / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(b)[i] = 0x3F800000u ^ (i & 0x7F);
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem)),
                 "r"(kTcN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid == 0) {
    // core matrices: 8 rows x 16 bytes, LBO 128 (K direction), SBO 256 (8-row groups)
    const uint64_t ad = desc_kmajor(smem_u32(a), 128, 256), bd = desc_kmajor(smem_u32(b), 128, 256);
    const uint32_t idesc = KIND == 0
        ? ((1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24))
        : ((1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24));
    for (int it = 0; it < iters; ++it) {
      const uint32_t acc = it == 0 ? 0u : 1u;
      if (KIND == 0)
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                     "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      else
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                     "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(&mbar)));
  }
  // bounded wait for the MMAs (every thread), then free the tensor memory
  uint32_t done = 0;
  for (int it = 0; it < (1 << 26) && !done; ++it)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(smem_u32(&mbar)), "r"(0));
  if (!done && tid == 0) atomicOr(failed, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN));
}

}  // namespace

// Returns 0 and *tflops on success, a negative value on a CUDA error or (tensor-core
// probes) a completion wait that gave up.
extern "C" int iedg_peak_probe(int kind, int reps, double* tflops) {
  if (!tflops || kind < 0 || kind > 4 || reps < 1) return -1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -2;
  void* buf = nullptr;
  int* failed = nullptr;
  if (cudaMalloc(&buf, 64) != cudaSuccess) return -2;
  if (cudaMalloc(&failed, sizeof(int)) != cudaSuccess || cudaMemset(failed, 0, sizeof(int)) != cudaSuccess) {
    cudaFree(buf);
    return -2;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double flop = 0.0;
  const int blocks_fma = sms * 8;
  auto launch = [&](bool timed) {
    const int r = timed ? reps : 1;
    switch (kind) {
      case 0: {
        const int iters = 2048 * r;
        k_fma<double><<<blocks_fma, kThreads>>>((double*)buf, iters, 1.0000001, 1e-9);
        flop = 2.0 * kChains * iters * (double)blocks_fma * kThreads;
      } break;
      case 1: {
        const int iters = 65536 * r;
        k_fma<float><<<blocks_fma, kThreads>>>((float*)buf, iters, 1.0000001f, 1e-9f);
        flop = 2.0 * kChains * iters * (double)blocks_fma * kThreads;
      } break;
      case 2: {
        const int iters = 1024 * r;
        k_dmma<<<blocks_fma, kThreads>>>((double*)buf, iters);
        flop = 2.0 * 8 * 8 * 4 * kChains * iters * (double)blocks_fma * (kThreads / 32);
      } break;
      case 3: {
        const int iters = 16384 * r;
        k_tcgen05<0><<<sms, 128>>>(iters, failed);
        flop = 2.0 * kTcM * kTcN * 8 * iters * (double)sms;
      } break;
      default: {
        const int iters = 16384 * r;
        k_tcgen05<1><<<sms, 128>>>(iters, failed);
        flop = 2.0 * kTcM * kTcN * 16 * iters * (double)sms;
      } break;
    }
  };
  launch(false);                                   // warm-up (clocks, first-launch costs)
  cudaEventRecord(e0);
  launch(true);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  int hf = 0;
  if (err == cudaSuccess) err = cudaMemcpy(&hf, failed, sizeof(int), cudaMemcpyDeviceToHost);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  cudaFree(failed);
  if (err != cudaSuccess) return -2;
  if (hf) return -3;
  *tflops = flop / (ms * 1e-3) / 1e12;
  return 0;
}
