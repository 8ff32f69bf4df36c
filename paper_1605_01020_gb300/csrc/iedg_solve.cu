// Trace solve K dU = R (Eq. LS) on the GPU: restarted GMRES with iterated classical
// Gram-Schmidt (two CGS passes per Arnoldi step) and left preconditioning
// M^-1 K dU = M^-1 R, as in the paper's parallel solver (Sec. 2.2.2).  On one GPU
// there is one subdomain; the preconditioner here is block Jacobi with the m x m
// diagonal blocks of K (the paper notes that zero overlap gives block Jacobi).
// The Hessenberg least-squares problem (Givens rotations) lives on the host; one
// small device-to-host copy per Arnoldi step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
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

// ---------------------------------------------------------------- BILU(0)
// Rows of one colour, one CTA per row: for each neighbour k eliminated before the row
// (in elimination order), L_ik = A_ik U_kk^-1, then A_ij -= L_ik U_kj for the row's
// later entries j present in row k (threads over j, binary search in row k); finally
// the inverse of the row's diagonal block.  Rows of one colour share no block.
constexpr int BI_THREADS = 128;
__device__ bool invert_block(int m, const double* __restrict__ a_in, double* __restrict__ out) {
  double a[5][10];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < 2 * m; ++j) a[i][j] = j < m ? a_in[i * m + j] : (j - m == i);
  for (int c = 0; c < m; ++c) {
    int pr = c;
    for (int r = c + 1; r < m; ++r)
      if (fabs(a[r][c]) > fabs(a[pr][c])) pr = r;
    if (a[pr][c] == 0.0) return false;
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
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) out[i * m + j] = a[i][m + j];
  return true;
}

__global__ void __launch_bounds__(BI_THREADS)
k_bilu_rows(int m, const int64_t* __restrict__ rows, const int64_t* __restrict__ row_ptr,
            const int32_t* __restrict__ col, const int32_t* __restrict__ ord, const int32_t* __restrict__ nlow,
            double* __restrict__ F, double* __restrict__ Uinv, int* __restrict__ flag) {
  __shared__ double Lb[25];
  const int tid = threadIdx.x, mm = m * m;
  const int64_t i = rows[blockIdx.x];
  const int64_t lo = row_ptr[i];
  const int len = (int)(row_ptr[i + 1] - lo);
  const int32_t* o = ord + lo;
  const int nl = nlow[i];
  for (int q = 0; q < nl; ++q) {
    const int64_t kk = lo + o[q];
    const int64_t k = col[kk];
    if (tid < mm) {
      const int r = tid / m, c = tid % m;
      double sacc = 0.0;
      for (int t = 0; t < m; ++t) sacc = fma(F[kk * mm + r * m + t], Uinv[k * mm + t * m + c], sacc);
      Lb[tid] = sacc;
    }
    __syncthreads();
    if (tid < mm) F[kk * mm + tid] = Lb[tid];
    const int64_t klo = row_ptr[k], khi = row_ptr[k + 1];
    for (int p = q + 1 + tid; p < len; p += BI_THREADS) {
      const int64_t jj = lo + o[p];
      const int32_t j = col[jj];
      int64_t a = klo, b = khi;
      while (a < b) {
        const int64_t mid = (a + b) >> 1;
        if (col[mid] < j) a = mid + 1; else b = mid;
      }
      if (a < khi && col[a] == j) {
        double* dst = F + jj * mm;
        const double* U = F + a * mm;
        for (int r = 0; r < m; ++r)
          for (int c = 0; c < m; ++c) {
            double sacc = dst[r * m + c];
            for (int t = 0; t < m; ++t) sacc = fma(-Lb[r * m + t], U[t * m + c], sacc);
            dst[r * m + c] = sacc;
          }
      }
    }
    __syncthreads();
  }
  if (tid == 0 && !invert_block(m, F + (lo + o[nl]) * mm, Uinv + i * mm)) atomicOr(flag, 1);
}

// Forward (lower) solve of the rows of one colour, one warp per row, in place:
// v_i -= sum_{k before i} L_ik v_k.
__global__ void k_bilu_fwd(int m, int64_t nrows, const int64_t* __restrict__ rows,
                           const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ ord, const int32_t* __restrict__ nlow,
                           const double* __restrict__ F, double* __restrict__ v) {
  const int lane = threadIdx.x & 31, mm = m * m;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= nrows) return;
  const int64_t i = rows[w], lo = row_ptr[i];
  const int32_t* o = ord + lo;
  const int nl = nlow[i];
  double acc[5] = {0, 0, 0, 0, 0};
  for (int q = lane; q < nl; q += 32) {
    const int64_t kk = lo + o[q];
    const double* blk = F + kk * mm;
    const double* x = v + (int64_t)col[kk] * m;
    for (int r = 0; r < m; ++r) {
      double sacc = 0.0;
      for (int t = 0; t < m; ++t) sacc = fma(blk[r * m + t], x[t], sacc);
      acc[r] += sacc;
    }
  }
  for (int r = 0; r < m; ++r)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off);
  if (lane < m) v[i * m + lane] -= acc[lane];
}

// Backward (upper) solve of the rows of one colour, in place:
// v_i = U_ii^-1 (v_i - sum_{j after i} U_ij v_j).
__global__ void k_bilu_bwd(int m, int64_t nrows, const int64_t* __restrict__ rows,
                           const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ ord, const int32_t* __restrict__ nlow,
                           const double* __restrict__ F, const double* __restrict__ Uinv, double* __restrict__ v) {
  const int lane = threadIdx.x & 31, mm = m * m;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= nrows) return;
  const int64_t i = rows[w], lo = row_ptr[i];
  const int len = (int)(row_ptr[i + 1] - lo);
  const int32_t* o = ord + lo;
  const int nl = nlow[i];
  double acc[5] = {0, 0, 0, 0, 0};
  for (int q = nl + 1 + lane; q < len; q += 32) {
    const int64_t kk = lo + o[q];
    const double* blk = F + kk * mm;
    const double* x = v + (int64_t)col[kk] * m;
    for (int r = 0; r < m; ++r) {
      double sacc = 0.0;
      for (int t = 0; t < m; ++t) sacc = fma(blk[r * m + t], x[t], sacc);
      acc[r] += sacc;
    }
  }
  for (int r = 0; r < m; ++r)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off);
  double sv[5];
  for (int t = 0; t < m; ++t) sv[t] = v[i * m + t] - acc[t];
  __syncwarp();
  if (lane < m) {
    double x = 0.0;
    for (int t = 0; t < m; ++t) x = fma(Uinv[(i * mm) + lane * m + t], sv[t], x);
    v[i * m + lane] = x;
  }
}

// ---------------------------------------------------------------- GMRES state on the device
// The Hessenberg column, Givens rotations, least-squares right-hand side and the
// residual estimate stay in device memory (kst below), so an Arnoldi step needs one
// host synchronisation (to read the residual estimate) instead of one per reduction.
// Layout of kst (doubles): h1 [R+1] | h2 [R+1] | H [(R+1) R] | cs [R] | sn [R] | g [R+1] |
// y [R] | scalars: hn2, beta, relres, done, jdone.
struct GmresState {
  double *h1, *h2, *H, *cs, *sn, *g, *y, *sc;
};
__host__ __device__ inline GmresState gmres_state(double* base) {
  constexpr int R = IEDG_MAX_RESTART;
  GmresState S;
  S.h1 = base;
  S.h2 = S.h1 + (R + 1);
  S.H = S.h2 + (R + 1);
  S.cs = S.H + (R + 1) * R;
  S.sn = S.cs + R;
  S.g = S.sn + R;
  S.y = S.g + (R + 1);
  S.sc = S.y + R;          // [0] hn2, [1] beta, [2] relres, [3] done, [4] jdone
  return S;
}

// y = x / sqrt(*n2), zero if *n2 == 0 (y may alias x)
__global__ void k_scale_norm(int64_t n, const double* __restrict__ n2, const double* x, double* y) {
  const double nn = *n2;
  const double a = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// start of a cycle: beta = sqrt(beta2), g = (beta, 0, ...), relres = beta / beta0, not done
__global__ void k_gmres_start(GmresState S, double beta0) {
  const double beta = sqrt(S.sc[0]);
  S.sc[1] = beta;
  for (int i = 0; i <= IEDG_MAX_RESTART; ++i) S.g[i] = 0.0;
  S.g[0] = beta;
  S.sc[2] = beta0 > 0.0 ? beta / beta0 : 0.0;
  S.sc[3] = 0.0;
}

// Hessenberg column j = h1 + h2 (the two Gram-Schmidt passes) with h_{j+1,j} = |w|;
// earlier rotations applied, a new one formed, g rotated, |g_{j+1}| / beta0 the
// residual estimate; done when it reaches rtol or the Krylov space is exhausted.
__global__ void k_gmres_givens(GmresState S, int j, double beta0, double rtol) {
  constexpr int R = IEDG_MAX_RESTART;
  double h[R + 1];
  for (int i = 0; i <= j; ++i) h[i] = S.h1[i] + S.h2[i];
  const double hn = sqrt(S.sc[0]);
  for (int i = 0; i < j; ++i) {
    const double a = S.cs[i] * h[i] + S.sn[i] * h[i + 1];
    const double b = -S.sn[i] * h[i] + S.cs[i] * h[i + 1];
    h[i] = a;
    h[i + 1] = b;
  }
  h[j + 1] = hn;
  const double r = hypot(h[j], h[j + 1]);
  S.cs[j] = r > 0.0 ? h[j] / r : 1.0;
  S.sn[j] = r > 0.0 ? h[j + 1] / r : 0.0;
  h[j] = r;
  S.g[j + 1] = -S.sn[j] * S.g[j];
  S.g[j] = S.cs[j] * S.g[j];
  for (int i = 0; i <= j; ++i) S.H[i * R + j] = h[i];
  const double rel = fabs(S.g[j + 1]) / beta0;
  S.sc[2] = rel;
  S.sc[3] = (rel <= rtol || hn == 0.0) ? 1.0 : 0.0;
}

// y = H(0:j, 0:j)^-1 g (upper triangular)
__global__ void k_gmres_backsolve(GmresState S, int j) {
  constexpr int R = IEDG_MAX_RESTART;
  for (int i = j - 1; i >= 0; --i) {
    double s = S.g[i];
    for (int k = i + 1; k < j; ++k) s -= S.H[i * R + k] * S.y[k];
    S.y[i] = s / S.H[i * R + i];
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

// Colouring and elimination orders of the trace pattern (host, once per handle).
static int bilu_setup(iedg_mesh* M, cudaStream_t st) {
  if (M->brows) return IEDG_OK;
  const int64_t T = M->T, nnzb = M->nnzb;
  std::vector<int64_t> rp(T + 1);
  std::vector<int32_t> col(nnzb);
  SV_TRY(cudaMemcpyAsync(rp.data(), M->row_ptr, (T + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SV_TRY(cudaMemcpyAsync(col.data(), M->col, nnzb * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SV_TRY(cudaStreamSynchronize(st));
  // greedy colouring in index order
  std::vector<int32_t> color(T, -1), mark;
  int32_t ncol = 0;
  for (int64_t t = 0; t < T; ++t) {
    mark.assign(ncol + 1, 0);
    for (int64_t k = rp[t]; k < rp[t + 1]; ++k)
      if (col[k] < t) mark[color[col[k]]] = 1;
    int32_t c = 0;
    while (mark[c]) ++c;
    color[t] = c;
    if (c + 1 > ncol) ncol = c + 1;
  }
  // rows sorted by (colour, index); rank = position in that order
  std::vector<int64_t> rows(T), cnt(ncol + 1, 0), rank(T);
  for (int64_t t = 0; t < T; ++t) cnt[color[t] + 1]++;
  for (int32_t c = 0; c < ncol; ++c) cnt[c + 1] += cnt[c];
  M->bcptr = cnt;
  {
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t t = 0; t < T; ++t) rows[fill[color[t]]++] = t;
  }
  for (int64_t r = 0; r < T; ++r) rank[rows[r]] = r;
  // per row: entries in elimination order, and how many come before the row
  std::vector<int32_t> ord(nnzb), nlow(T);
  for (int64_t t = 0; t < T; ++t) {
    const int64_t lo = rp[t];
    const int32_t len = (int32_t)(rp[t + 1] - lo);
    int32_t* o = ord.data() + lo;
    for (int32_t q = 0; q < len; ++q) o[q] = q;
    std::sort(o, o + len, [&](int32_t a, int32_t b) { return rank[col[lo + a]] < rank[col[lo + b]]; });
    int32_t nl = 0;
    while (nl < len && rank[col[lo + o[nl]]] < rank[t]) ++nl;
    nlow[t] = nl;
  }
  auto put = [&](auto** dst, const auto& h) -> cudaError_t {
    using E = typename std::remove_const<typename std::remove_reference<decltype(h[0])>::type>::type;
    E* d = nullptr;
    cudaError_t e = cudaMalloc((void**)&d, std::max<size_t>(h.size(), 1) * sizeof(E));
    if (e != cudaSuccess) return e;
    M->allocs.push_back(d);
    M->ws_bytes += (int64_t)(h.size() * sizeof(E));
    *dst = d;
    return cudaMemcpyAsync(d, h.data(), h.size() * sizeof(E), cudaMemcpyHostToDevice, st);
  };
  SV_TRY(put(&M->brows, rows));
  SV_TRY(put(&M->bord, ord));
  SV_TRY(put(&M->bnlow, nlow));
  SV_TRY(cudaStreamSynchronize(st));
  M->bcolor = color;
  return IEDG_OK;
}

static int bilu_factor(iedg_mesh* M, const double* K, double* F, cudaStream_t st) {
  int rc = bilu_setup(M, st);
  if (rc != IEDG_OK) return rc;
  const int m = M->dm.m;
  if (F != K) SV_TRY(cudaMemcpyAsync(F, K, (size_t)M->nnzb * m * m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SV_TRY(cudaMemsetAsync(M->dev_flag, 0, sizeof(int), st));
  for (size_t c = 0; c + 1 < M->bcptr.size(); ++c) {
    const int64_t nr = M->bcptr[c + 1] - M->bcptr[c];
    if (nr == 0) continue;
    SV_TRY((k_bilu_rows<<<(unsigned)nr, BI_THREADS, 0, st>>>(m, M->brows + M->bcptr[c], M->row_ptr, M->col, M->bord,
                                                             M->bnlow, F, M->dinv, M->dev_flag),
            cudaGetLastError()));
  }
  int flag = 0;
  SV_TRY(cudaMemcpyAsync(&flag, M->dev_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  SV_TRY(cudaStreamSynchronize(st));
  if (flag) {
    M->err = "BILU(0): singular pivot block";
    return IEDG_ERR_INVALID_ARG;
  }
  return IEDG_OK;
}

// v <- U^-1 L^-1 v, colour by colour (one launch per colour and sweep: a single-block
// form of all colours was measured slower, one SM's bandwidth for the whole factor)
static cudaError_t bilu_apply(iedg_mesh* M, const double* F, double* v, cudaStream_t st) {
  const int m = M->dm.m;
  const size_t nc = M->bcptr.size() - 1;

  for (size_t c = 0; c < nc; ++c) {
    const int64_t nr = M->bcptr[c + 1] - M->bcptr[c];
    if (nr == 0) continue;
    k_bilu_fwd<<<(unsigned)((nr * 32 + SV_THREADS - 1) / SV_THREADS), SV_THREADS, 0, st>>>(
        m, nr, M->brows + M->bcptr[c], M->row_ptr, M->col, M->bord, M->bnlow, F, v);
  }
  for (size_t c = nc; c-- > 0;) {
    const int64_t nr = M->bcptr[c + 1] - M->bcptr[c];
    if (nr == 0) continue;
    k_bilu_bwd<<<(unsigned)((nr * 32 + SV_THREADS - 1) / SV_THREADS), SV_THREADS, 0, st>>>(
        m, nr, M->brows + M->bcptr[c], M->row_ptr, M->col, M->bord, M->bnlow, F, M->dinv, v);
  }
  return cudaGetLastError();
}

extern "C" int iedg_set_trace_precond(iedg_mesh* M, int32_t kind) {
  if (!M) return IEDG_ERR_INVALID_ARG;
  if (kind != IEDG_PREC_BLOCK_JACOBI && kind != IEDG_PREC_BILU0) {
    M->err = "iedg_set_trace_precond: unknown preconditioner";
    return IEDG_ERR_INVALID_ARG;
  }
  M->prec_kind = kind;
  return IEDG_OK;
}

extern "C" int iedg_bilu0_factor(iedg_mesh* M, const double* K, double* F, void* stream) {
  if (!M || !K || !F) {
    if (M) M->err = "iedg_bilu0_factor: null argument";
    return IEDG_ERR_INVALID_ARG;
  }
  return bilu_factor(M, K, F, (cudaStream_t)stream);
}

extern "C" int iedg_bilu0_apply(iedg_mesh* M, const double* F, const double* r, double* x, void* stream) {
  if (!M || !F || !r || !x) {
    if (M) M->err = "iedg_bilu0_apply: null argument";
    return IEDG_ERR_INVALID_ARG;
  }
  if (!M->brows) {
    M->err = "iedg_bilu0_apply: no factorisation on this handle";
    return IEDG_ERR_NOT_ASSEMBLED;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (x != r) SV_TRY(cudaMemcpyAsync(x, r, (size_t)M->T * M->dm.m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SV_TRY(bilu_apply(M, F, x, st));
  return IEDG_OK;
}

extern "C" int iedg_trace_colors(iedg_mesh* M, int32_t* colors) {
  if (!M || !colors) return IEDG_ERR_INVALID_ARG;
  int rc = bilu_setup(M, 0);
  if (rc != IEDG_OK) return rc;
  std::memcpy(colors, M->bcolor.data(), M->bcolor.size() * sizeof(int32_t));
  return IEDG_OK;
}

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
  const unsigned g = grid_for(n);
  const unsigned gw = (unsigned)((T * 32 + SV_THREADS - 1) / SV_THREADS);
  const bool bilu = M->prec_kind == IEDG_PREC_BILU0;
  if (bilu) {
    if (!M->bf) {
      double* f = nullptr;
      SV_TRY(cudaMalloc(&f, (size_t)M->nnzb * m * m * sizeof(double)));
      M->allocs.push_back(f);
      M->ws_bytes += (int64_t)M->nnzb * m * m * sizeof(double);
      M->bf = f;
    }
    int rc = bilu_factor(M, K, M->bf, st);
    if (rc != IEDG_OK) return rc;
  }
  // y = M^-1 x (in place allowed)
  auto prec = [&](const double* x, double* y) -> cudaError_t {
    if (!bilu) {
      k_prec<<<(unsigned)((T + 127) / 128), 128, 0, st>>>(m, T, Dinv, x, y);
      return cudaGetLastError();
    }
    if (x != y) {
      cudaError_t e = cudaMemcpyAsync(y, x, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
    return bilu_apply(M, M->bf, y, st);
  };
  SV_TRY(cudaMemsetAsync(M->dev_flag, 0, sizeof(int), st));
  if (!bilu)
    SV_TRY((k_diag_inv<<<(unsigned)((T + 127) / 128), 128, 0, st>>>(m, T, M->row_ptr, M->col, K, Dinv, M->dev_flag),
            cudaGetLastError()));
  // sums of products into device memory (fixed block order: deterministic)
  auto dots_dev = [&](int nv, const double* Vb, const double* x, double* out_dev) -> cudaError_t {
    k_dots<<<SV_PART, SV_THREADS, 0, st>>>(n, nv, Vb, x, part);
    k_sum_partials<<<1, 64, 0, st>>>(nv, part, out_dev);
    return cudaGetLastError();
  };
  const GmresState S = gmres_state(M->kst);
  // the host reads three scalars of the device state: squared norm, residual estimate, done
  auto read_state = [&](double* out3) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(out3, S.sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  };
  // x0 = 0, r0 = M^-1 R
  SV_TRY(cudaMemsetAsync(dU, 0, n * sizeof(double), st));
  SV_TRY(prec(R, V));
  SV_TRY(dots_dev(1, V, V, S.sc));
  double hs[4] = {0, 0, 0, 0};
  SV_TRY(read_state(hs));
  const double beta0 = std::sqrt(hs[0]);
  int flag = 0;
  SV_TRY(cudaMemcpy(&flag, M->dev_flag, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    M->err = "iedg_trace_solve: singular diagonal block of K";
    return IEDG_ERR_INVALID_ARG;
  }
  int total = 0;
  double relres = beta0 > 0.0 ? 1.0 : 0.0;
  bool first = true;
  while (beta0 > 0.0 && total < max_iter && relres > rtol) {
    if (!first) {
      // r = M^-1 (R - K x)
      SV_TRY((k_spmv<<<gw, SV_THREADS, 0, st>>>(m, T, M->row_ptr, M->col, K, Dinv, dU, tmp, false), cudaGetLastError()));
      SV_TRY((k_residual<<<g, SV_THREADS, 0, st>>>(m, n, R, tmp, tmp), cudaGetLastError()));
      SV_TRY(prec(tmp, V));
      SV_TRY(dots_dev(1, V, V, S.sc));
    }
    SV_TRY((k_gmres_start<<<1, 1, 0, st>>>(S, beta0), cudaGetLastError()));
    if (!first) {
      SV_TRY(read_state(hs));
      relres = hs[2];
      if (relres <= rtol) break;
    }
    first = false;
    SV_TRY((k_scale_norm<<<g, SV_THREADS, 0, st>>>(n, S.sc, V, V), cudaGetLastError()));
    int j = 0;
    for (; j < restart && total < max_iter; ++j, ++total) {
      double* vj = V + (int64_t)j * n;
      double* vn = V + (int64_t)(j + 1) * n;
      SV_TRY((k_spmv<<<gw, SV_THREADS, 0, st>>>(m, T, M->row_ptr, M->col, K, Dinv, vj, w, !bilu), cudaGetLastError()));
      if (bilu) SV_TRY(prec(w, w));
      // iterated classical Gram-Schmidt: two passes, coefficients kept on the device
      SV_TRY(dots_dev(j + 1, V, w, S.h1));
      SV_TRY((k_orth<<<g, SV_THREADS, 0, st>>>(n, j + 1, V, S.h1, w), cudaGetLastError()));
      SV_TRY(dots_dev(j + 1, V, w, S.h2));
      SV_TRY((k_orth<<<g, SV_THREADS, 0, st>>>(n, j + 1, V, S.h2, w), cudaGetLastError()));
      SV_TRY(dots_dev(1, w, w, S.sc));
      SV_TRY((k_scale_norm<<<g, SV_THREADS, 0, st>>>(n, S.sc, w, vn), cudaGetLastError()));
      SV_TRY((k_gmres_givens<<<1, 1, 0, st>>>(S, j, beta0, rtol), cudaGetLastError()));
      SV_TRY(read_state(hs));                         // the one synchronisation of the step
      relres = hs[2];
      if (hs[3] != 0.0) { ++j; ++total; break; }
    }
    // y = H(0:j, 0:j)^-1 g, x += V y
    SV_TRY((k_gmres_backsolve<<<1, 1, 0, st>>>(S, j), cudaGetLastError()));
    SV_TRY((k_update<<<g, SV_THREADS, 0, st>>>(n, j, V, S.y, dU), cudaGetLastError()));
  }
  SV_TRY(cudaStreamSynchronize(st));
  if (iterations) *iterations = total;
  if (rel_residual) *rel_residual = relres;
  return IEDG_OK;
}
