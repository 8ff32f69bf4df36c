// Trace solve K dU = R (Eq. LS) on the GPU: restarted GMRES with iterated classical
// Gram-Schmidt (two CGS passes per Arnoldi step) and left preconditioning
// M^-1 K dU = M^-1 R, as in the paper's parallel solver (Sec. 2.2.2).  On one GPU
// there is one subdomain; the preconditioner here is block Jacobi with the m x m
// diagonal blocks of K (the paper notes that zero overlap gives block Jacobi).
// The Hessenberg least-squares problem (Givens rotations) lives on the host; one
// small device-to-host copy per Arnoldi step.
#include <cmath>
#include <cstring>
#include <vector>

#include "iedg_internal.cuh"

using namespace iedg;

namespace {

constexpr int SV_THREADS = 256;
constexpr int SV_PART = 512;        // CTAs of the dot-product kernels

// Dinv[t] = inverse of the diagonal block K[t][t] (Gauss-Jordan, partial pivoting).
__global__ void k_diag_inv(int m, int64_t T, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const double* __restrict__ K, double* __restrict__ Dinv, int* __restrict__ flag) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  int64_t lo = row_ptr[t], hi = row_ptr[t + 1], blk = -1;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (col[mid] < t) lo = mid + 1; else hi = mid;
  }
  if (lo < row_ptr[t + 1] && col[lo] == t) blk = lo;
  double a[5][10];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < 2 * m; ++j) a[i][j] = j < m ? (blk >= 0 ? K[(blk * m + i) * m + j] : 0.0) : (j - m == i);
  bool ok = blk >= 0;
  for (int c = 0; c < m && ok; ++c) {
    int pr = c;
    for (int r = c + 1; r < m; ++r)
      if (fabs(a[r][c]) > fabs(a[pr][c])) pr = r;
    if (a[pr][c] == 0.0) { ok = false; break; }
    if (pr != c)
      for (int j = 0; j < 2 * m; ++j) { double x = a[c][j]; a[c][j] = a[pr][j]; a[pr][j] = x; }
    double inv = 1.0 / a[c][c];
    for (int j = 0; j < 2 * m; ++j) a[c][j] *= inv;
    for (int r = 0; r < m; ++r) {
      if (r == c) continue;
      double f = a[r][c];
      for (int j = 0; j < 2 * m; ++j) a[r][j] -= f * a[c][j];
    }
  }
  if (!ok) atomicOr(flag, 1);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Dinv[(t * m + i) * m + j] = ok ? a[i][m + j] : (i == j);
}

// y = M^-1 (K x) (prec = true) or y = K x; one warp per block row.
__global__ void k_spmv(int m, int64_t T, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                       const double* __restrict__ K, const double* __restrict__ Dinv, const double* __restrict__ x,
                       double* __restrict__ y, bool prec) {
  const int lane = threadIdx.x & 31;
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (t >= T) return;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int64_t b = row_ptr[t] + lane; b < row_ptr[t + 1]; b += 32) {
    const double* blk = K + b * m * m;
    const double* xc = x + (int64_t)col[b] * m;
    for (int i = 0; i < m; ++i) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s = fma(blk[i * m + k], xc[k], s);
      acc[i] += s;
    }
  }
  for (int i = 0; i < m; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
  if (lane < m) {
    double v;
    if (prec) {
      v = 0.0;
      for (int k = 0; k < m; ++k) v = fma(Dinv[(t * m + lane) * m + k], acc[k], v);
    } else {
      v = acc[lane];
    }
    y[t * m + lane] = v;
  }
}

// partial[v * SV_PART + blk] = sum over the block's slice of V[v] . w, v < nv
__global__ void k_dots(int64_t n, int nv, const double* __restrict__ V, const double* __restrict__ w,
                       double* __restrict__ partial) {
  __shared__ double red[SV_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int v = 0; v < nv; ++v) {
    const double* a = V + (int64_t)v * n;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * SV_THREADS + tid; i < n; i += (int64_t)gridDim.x * SV_THREADS)
      s = fma(a[i], w[i], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int k = 0; k < SV_THREADS / 32; ++k) t += red[k];
      partial[(int64_t)v * SV_PART + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// out[v] = sum_blk partial[v][blk] (fixed order: deterministic)
__global__ void k_sum_partials(int nv, const double* __restrict__ partial, double* __restrict__ out) {
  const int v = threadIdx.x;
  if (v >= nv) return;
  double s = 0.0;
  for (int b = 0; b < SV_PART; ++b) s += partial[(int64_t)v * SV_PART + b];
  out[v] = s;
}

// w -= sum_v h[v] V[v]
__global__ void k_orth(int64_t n, int nv, const double* __restrict__ V, const double* __restrict__ h,
                       double* __restrict__ w) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int v = 0; v < nv; ++v) s = fma(-h[v], V[(int64_t)v * n + i], s);
    w[i] = s;
  }
}

// y = a x (y may alias x)
__global__ void k_scale(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// x += sum_v c[v] V[v]
__global__ void k_update(int64_t n, int nv, const double* __restrict__ V, const double* __restrict__ c,
                         double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = x[i];
    for (int v = 0; v < nv; ++v) s = fma(c[v], V[(int64_t)v * n + i], s);
    x[i] = s;
  }
}

// r = b - K x, then r <- M^-1 r (in place into r)
__global__ void k_residual(int m, int64_t n, const double* __restrict__ b, const double* __restrict__ Kx,
                           double* __restrict__ r) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - Kx[i];
}

// y = M^-1 x (block Jacobi), one thread per block row
__global__ void k_prec(int m, int64_t T, const double* __restrict__ Dinv, const double* __restrict__ x,
                       double* __restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  double xs[5];
  for (int k = 0; k < m; ++k) xs[k] = x[t * m + k];
  for (int i = 0; i < m; ++i) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) s = fma(Dinv[(t * m + i) * m + k], xs[k], s);
    y[t * m + i] = s;
  }
}

unsigned grid_for(int64_t n) {
  int64_t g = (n + SV_THREADS - 1) / SV_THREADS;
  return (unsigned)(g < 4096 ? g : 4096);
}

}  // namespace

#define SV_TRY(call)                                                                       \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      M->err = std::string("iedg_trace_solve: ") + #call + ": " + cudaGetErrorString(e_); \
      return IEDG_ERR_CUDA;                                                                \
    }                                                                                      \
  } while (0)

extern "C" int iedg_trace_solve(iedg_mesh* M, const double* K, const double* R, double* dU, int32_t restart,
                                int32_t max_iter, double rtol, int32_t* iterations, double* rel_residual,
                                void* stream) {
  if (!M || !K || !R || !dU) {
    if (M) M->err = "iedg_trace_solve: null argument";
    return IEDG_ERR_INVALID_ARG;
  }
  if (restart < 1 || restart > IEDG_MAX_RESTART || max_iter < 1 || !(rtol > 0.0)) {
    M->err = "iedg_trace_solve: restart must be 1..IEDG_MAX_RESTART, max_iter >= 1, rtol > 0";
    return IEDG_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int m = M->dm.m;
  const int64_t T = M->T, n = T * m;
  double* V = M->kry;                     // [restart+1][n]
  double* w = V + (int64_t)(IEDG_MAX_RESTART + 1) * n;
  double* tmp = w + n;
  double* Dinv = M->dinv;
  double* part = M->kpart;                // [restart+1][SV_PART]
  double* hdev = M->khdev;                // [restart+1]
  const unsigned g = grid_for(n);
  const unsigned gw = (unsigned)((T * 32 + SV_THREADS - 1) / SV_THREADS);
  SV_TRY(cudaMemsetAsync(M->dev_flag, 0, sizeof(int), st));
  SV_TRY((k_diag_inv<<<(unsigned)((T + 127) / 128), 128, 0, st>>>(m, T, M->row_ptr, M->col, K, Dinv, M->dev_flag),
          cudaGetLastError()));
  auto dots = [&](int nv, const double* Vb, const double* x, double* out_host) -> cudaError_t {
    k_dots<<<SV_PART, SV_THREADS, 0, st>>>(n, nv, Vb, x, part);
    k_sum_partials<<<1, 64, 0, st>>>(nv, part, hdev);
    cudaError_t e = cudaMemcpyAsync(out_host, hdev, nv * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  };
  // x0 = 0, r0 = M^-1 R
  SV_TRY(cudaMemsetAsync(dU, 0, n * sizeof(double), st));
  SV_TRY((k_prec<<<(unsigned)((T + 127) / 128), 128, 0, st>>>(m, T, Dinv, R, V), cudaGetLastError()));
  double beta0 = 0.0;
  SV_TRY(dots(1, V, V, &beta0));
  beta0 = std::sqrt(beta0);
  int flag = 0;
  SV_TRY(cudaMemcpy(&flag, M->dev_flag, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    M->err = "iedg_trace_solve: singular diagonal block of K";
    return IEDG_ERR_INVALID_ARG;
  }
  int total = 0;
  double relres = beta0 > 0.0 ? 1.0 : 0.0;
  std::vector<double> H((restart + 1) * restart), cs(restart), sn(restart), gvec(restart + 1), h(restart + 1),
      h2(restart + 1), y(restart);
  double beta = beta0;
  bool first = true;
  while (beta0 > 0.0 && total < max_iter && relres > rtol) {
    if (!first) {
      // r = M^-1 (R - K x)
      SV_TRY((k_spmv<<<gw, SV_THREADS, 0, st>>>(m, T, M->row_ptr, M->col, K, Dinv, dU, tmp, false), cudaGetLastError()));
      SV_TRY((k_residual<<<g, SV_THREADS, 0, st>>>(m, n, R, tmp, tmp), cudaGetLastError()));
      SV_TRY((k_prec<<<(unsigned)((T + 127) / 128), 128, 0, st>>>(m, T, Dinv, tmp, V), cudaGetLastError()));
      double bb = 0.0;
      SV_TRY(dots(1, V, V, &bb));
      beta = std::sqrt(bb);
      relres = beta / beta0;
      if (relres <= rtol) break;
    }
    first = false;
    SV_TRY((k_scale<<<g, SV_THREADS, 0, st>>>(n, 1.0 / beta, V, V), cudaGetLastError()));
    std::fill(gvec.begin(), gvec.end(), 0.0);
    gvec[0] = beta;
    int j = 0;
    for (; j < restart && total < max_iter; ++j, ++total) {
      double* vj = V + (int64_t)j * n;
      double* vn = V + (int64_t)(j + 1) * n;
      SV_TRY((k_spmv<<<gw, SV_THREADS, 0, st>>>(m, T, M->row_ptr, M->col, K, Dinv, vj, w, true), cudaGetLastError()));
      // iterated classical Gram-Schmidt: two passes
      SV_TRY(dots(j + 1, V, w, h.data()));
      SV_TRY(cudaMemcpyAsync(hdev, h.data(), (j + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
      SV_TRY((k_orth<<<g, SV_THREADS, 0, st>>>(n, j + 1, V, hdev, w), cudaGetLastError()));
      SV_TRY(dots(j + 1, V, w, h2.data()));
      SV_TRY(cudaMemcpyAsync(hdev, h2.data(), (j + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
      SV_TRY((k_orth<<<g, SV_THREADS, 0, st>>>(n, j + 1, V, hdev, w), cudaGetLastError()));
      for (int i = 0; i <= j; ++i) h[i] += h2[i];
      double hn = 0.0;
      SV_TRY(dots(1, w, w, &hn));
      hn = std::sqrt(hn);
      SV_TRY((k_scale<<<g, SV_THREADS, 0, st>>>(n, hn > 0.0 ? 1.0 / hn : 0.0, w, vn), cudaGetLastError()));
      // apply previous rotations, then a new one
      for (int i = 0; i < j; ++i) {
        double a = cs[i] * h[i] + sn[i] * h[i + 1];
        double b = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = a;
        h[i + 1] = b;
      }
      h[j + 1] = hn;
      double r = std::hypot(h[j], h[j + 1]);
      cs[j] = r > 0.0 ? h[j] / r : 1.0;
      sn[j] = r > 0.0 ? h[j + 1] / r : 0.0;
      h[j] = r;
      h[j + 1] = 0.0;
      gvec[j + 1] = -sn[j] * gvec[j];
      gvec[j] = cs[j] * gvec[j];
      for (int i = 0; i <= j; ++i) H[i * restart + j] = h[i];
      relres = std::fabs(gvec[j + 1]) / beta0;
      if (relres <= rtol || hn == 0.0) { ++j; ++total; break; }
    }
    // y = H(0:j, 0:j)^-1 g, x += V y
    for (int i = j - 1; i >= 0; --i) {
      double s = gvec[i];
      for (int k = i + 1; k < j; ++k) s -= H[i * restart + k] * y[k];
      y[i] = s / H[i * restart + i];
    }
    SV_TRY(cudaMemcpyAsync(hdev, y.data(), j * sizeof(double), cudaMemcpyHostToDevice, st));
    SV_TRY((k_update<<<g, SV_THREADS, 0, st>>>(n, j, V, hdev, dU), cudaGetLastError()));
    SV_TRY(cudaStreamSynchronize(st));
  }
  if (iterations) *iterations = total;
  if (rel_residual) *rel_residual = relres;
  return IEDG_OK;
}
