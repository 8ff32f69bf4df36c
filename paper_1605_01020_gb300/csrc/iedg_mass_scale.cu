// Scaling of the element system by the element mass matrix before the low-precision
// factorisation (mixed forms, handle flag IEDG_FLAG_MASS_SCALING).
//
// The u-block of the q-eliminated element system is dominated by the implicit
// stage's alpha M (Eq. IEDG b with the DIRK mass term) and inherits the conditioning
// of the mass matrix.  With M = L L^T (Cholesky) and S = I_m (x) L^-1 (one block per
// conserved component of the component-major u-unknowns), the bordered matrix becomes
//     [ S A~ S^T   S B~   S F~ ]
//     [ C~ S^T     D~     G~   ],
// whose Schur complement is the same K = D~ - C~ A~^-1 B~ (Eq. LS) and whose u-block
// S A~ S^T ~ alpha I + ... is far better conditioned; the u-unknowns of the scaled
// system are S^-T du.  The refinement solves A~ x = b as x = S^T (S A~ S^T)^-1 S b with
// the factors of the scaled matrix and FP64 residuals of the unscaled operator.
//
// Per mesh: k_mass_chol forms L^-1 in FP64 and keeps it in FP32 (lower triangular).
// Per assembly: k_scale_rows applies S from the left to the u-rows, k_scale_cols S^T
// from the right to the u-columns of every row.
#include "iedg_internal.cuh"

namespace iedg {
namespace {

constexpr int MS_THREADS = 256;

// L^-1 of the element's mass matrix.  Cholesky in place (lower triangle of Ls), then
// column c of X = L^-1 by forward substitution in thread c, kept in the strict upper
// triangle of Ls (X[i][c] at Ls[c][i]) and its diagonal in xd.
__global__ void __launch_bounds__(MS_THREADS) k_mass_chol(int Np, const double* __restrict__ Mass,
                                                          float* __restrict__ Linv32, int* __restrict__ flag) {
  extern __shared__ double ls[];
  double* xd = ls + (size_t)Np * Np;
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  const double* M = Mass + (size_t)e * Np * Np;
  for (int i = tid; i < Np * Np; i += MS_THREADS) ls[i] = M[i];
  __syncthreads();
  for (int j = 0; j < Np; ++j) {
    if (tid == 0) {
      const double d = ls[j * Np + j];
      if (!(d > 0.0)) atomicOr(flag, 2);
      ls[j * Np + j] = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    const double dj = ls[j * Np + j];
    for (int i = j + 1 + tid; i < Np; i += MS_THREADS) ls[i * Np + j] /= dj;
    __syncthreads();
    // lower trailing update A[i][k] -= L[i][j] L[k][j] for j < k <= i
    const int rem = Np - j - 1;
    for (int idx = tid; idx < rem * rem; idx += MS_THREADS) {
      const int i = j + 1 + idx / rem, k = j + 1 + idx % rem;
      if (k <= i) ls[i * Np + k] = fma(-ls[i * Np + j], ls[k * Np + j], ls[i * Np + k]);
    }
    __syncthreads();
  }
  for (int c = tid; c < Np; c += MS_THREADS) {
    xd[c] = 1.0 / ls[c * Np + c];
    for (int i = c + 1; i < Np; ++i) {
      double s = ls[i * Np + c] * xd[c];
      for (int k = c + 1; k < i; ++k) s = fma(ls[i * Np + k], ls[c * Np + k], s);
      ls[c * Np + i] = -s / ls[i * Np + i];
    }
  }
  __syncthreads();
  float* out = Linv32 + (size_t)e * Np * Np;
  for (int idx = tid; idx < Np * Np; idx += MS_THREADS) {
    const int i = idx / Np, c = idx % Np;
    out[idx] = i < c ? 0.f : (float)(i == c ? xd[c] : ls[c * Np + i]);
  }
}

constexpr int MS_CH = 64;     // columns (rows) per staged chunk
constexpr int MS_T = 4;       // register tile MS_T x MS_T per thread

// u-rows of component i: R_i <- L^-1 R_i over all n + 1 columns (L^-1 is stored with
// zeros above its diagonal, so the tile sums simply stop at the tile's last row).
__global__ void __launch_bounds__(MS_THREADS) k_scale_rows(Dims dm, const float* __restrict__ Linv32,
                                                           float* __restrict__ S) {
  extern __shared__ float fs[];
  const int Np = dm.Np, ncol = dm.n + 1;
  const int64_t e = blockIdx.x / dm.m;
  const int i = blockIdx.x % dm.m, tid = threadIdx.x;
  const int sp = Np + 1;
  float* Li = fs;                      // [Np][Np + 1]
  float* st = Li + ((Np * sp + 3) & ~3);   // [Np][MS_CH], 16-byte aligned (float4 reads)
  const float* L = Linv32 + (size_t)e * Np * Np;
  for (int q = tid; q < Np * Np; q += MS_THREADS) Li[(q / Np) * sp + q % Np] = L[q];
  float* R = S + (e * (int64_t)dm.n + (int64_t)i * Np) * dm.ld;
  const int rt = (Np + MS_T - 1) / MS_T, ct = MS_CH / MS_T;
  for (int c0 = 0; c0 < ncol; c0 += MS_CH) {
    __syncthreads();
    for (int q = tid; q < Np * MS_CH; q += MS_THREADS) {
      const int b = q / MS_CH, c = q % MS_CH;
      st[q] = c0 + c < ncol ? R[(int64_t)b * dm.ld + c0 + c] : 0.f;
    }
    __syncthreads();
    for (int tq = tid; tq < rt * ct; tq += MS_THREADS) {
      const int a0 = (tq / ct) * MS_T, cc = (tq % ct) * MS_T;
      float acc[MS_T][MS_T] = {};
      const int bend = min(Np, a0 + MS_T);
      for (int b = 0; b < bend; ++b) {
        float lv[MS_T];
#pragma unroll
        for (int x = 0; x < MS_T; ++x) lv[x] = a0 + x < Np ? Li[(a0 + x) * sp + b] : 0.f;
        const float4 sv = *reinterpret_cast<const float4*>(st + b * MS_CH + cc);
#pragma unroll
        for (int x = 0; x < MS_T; ++x) {
          acc[x][0] = fmaf(lv[x], sv.x, acc[x][0]);
          acc[x][1] = fmaf(lv[x], sv.y, acc[x][1]);
          acc[x][2] = fmaf(lv[x], sv.z, acc[x][2]);
          acc[x][3] = fmaf(lv[x], sv.w, acc[x][3]);
        }
      }
#pragma unroll
      for (int x = 0; x < MS_T; ++x)
#pragma unroll
        for (int y = 0; y < MS_T; ++y)
          if (a0 + x < Np && c0 + cc + y < ncol) R[(int64_t)(a0 + x) * dm.ld + c0 + cc + y] = acc[x][y];
    }
  }
}

// u-columns of component k in every row: C_k <- C_k L^-T.
__global__ void __launch_bounds__(MS_THREADS) k_scale_cols(Dims dm, const float* __restrict__ Linv32,
                                                           float* __restrict__ S) {
  extern __shared__ float fs[];
  const int Np = dm.Np, n = dm.n;
  const int64_t e = blockIdx.x / dm.m;
  const int k = blockIdx.x % dm.m, tid = threadIdx.x;
  // L^-1 with its rows padded to Np + 1 values (conflict-free column reads)
  const int sp = Np + 1;
  float* Li = fs;                      // [Np][Np + 1]
  float* st = Li + Np * sp;            // [MS_CH][Np + 1]
  const float* L = Linv32 + (size_t)e * Np * Np;
  for (int q = tid; q < Np * Np; q += MS_THREADS) Li[(q / Np) * sp + q % Np] = L[q];
  float* C = S + e * (int64_t)n * dm.ld + (int64_t)k * Np;
  const int at = (Np + MS_T - 1) / MS_T, rt = MS_CH / MS_T;
  for (int r0 = 0; r0 < n; r0 += MS_CH) {
    __syncthreads();
    for (int q = tid; q < MS_CH * Np; q += MS_THREADS) {
      const int r = q / Np, b = q % Np;
      st[r * sp + b] = r0 + r < n ? C[(int64_t)(r0 + r) * dm.ld + b] : 0.f;
    }
    __syncthreads();
    for (int tq = tid; tq < rt * at; tq += MS_THREADS) {
      const int rr = (tq / at) * MS_T, a0 = (tq % at) * MS_T;
      float acc[MS_T][MS_T] = {};
      const int bend = min(Np, a0 + MS_T);
      for (int b = 0; b < bend; ++b) {
        float sv[MS_T], lv[MS_T];
#pragma unroll
        for (int x = 0; x < MS_T; ++x) {
          sv[x] = st[(rr + x) * sp + b];
          lv[x] = a0 + x < Np ? Li[(a0 + x) * sp + b] : 0.f;
        }
#pragma unroll
        for (int x = 0; x < MS_T; ++x)
#pragma unroll
          for (int y = 0; y < MS_T; ++y) acc[x][y] = fmaf(sv[x], lv[y], acc[x][y]);
      }
#pragma unroll
      for (int x = 0; x < MS_T; ++x)
#pragma unroll
        for (int y = 0; y < MS_T; ++y)
          if (r0 + rr + x < n && a0 + y < Np) C[(int64_t)(r0 + rr + x) * dm.ld + a0 + y] = acc[x][y];
    }
  }
}

}  // namespace

cudaError_t launch_mass_chol(iedg_mesh* M, cudaStream_t st) {
  const int Np = M->dm.Np;
  const size_t smem = sizeof(double) * ((size_t)Np * Np + Np);
  cudaError_t err = cudaFuncSetAttribute(k_mass_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_mass_chol<<<(unsigned)M->E, MS_THREADS, smem, st>>>(Np, M->geo.Mass, M->Linv32, M->dev_flag);
  return cudaGetLastError();
}

cudaError_t launch_mass_scale(iedg_mesh* M, cudaStream_t st) {
  const Dims& dm = M->dm;
  const size_t s1 = sizeof(float) * (((size_t)dm.Np * (dm.Np + 1) + 3) / 4 * 4 + (size_t)dm.Np * MS_CH);
  const size_t s2 = sizeof(float) * ((size_t)dm.Np * (dm.Np + 1) + (size_t)MS_CH * (dm.Np + 1));
  cudaError_t err = cudaFuncSetAttribute(k_scale_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_scale_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2);
  if (err != cudaSuccess) return err;
  const unsigned grid = (unsigned)(M->E * dm.m);
  k_scale_rows<<<grid, MS_THREADS, s1, st>>>(dm, M->Linv32, M->S32);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_scale_cols<<<grid, MS_THREADS, s2, st>>>(dm, M->Linv32, M->S32);
  return cudaGetLastError();
}

}  // namespace iedg
