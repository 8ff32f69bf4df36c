// Assembly of the condensed element matrices into the block compressed-row trace
// matrix, K = sum_e P_e^T K_e P_e, R = sum_e P_e^T R_e (Sec. 2.2.2: m x m blocks),
// as a deterministic gather over precomputed contribution lists (element order),
// and the element back-substitution dZ_e = A_e^-1 (F_e - B_e dU_e).
#include "iedg_internal.cuh"

namespace iedg {
namespace {

// One thread per (block, i, k) entry; S is the FP64 or the FP32 element matrix.
// Contributions are packed as (e P + s) P + t, P = Nb (uniform meshes) or the slot
// stride of meshes with mixed orders, whose matrices have per-element sizes (lud).
// With an FP64 fallback in use (fb_count > 0), elements that have a slot contribute
// their FP64 block from the slot matrices fbS instead.
template <class T>
__global__ void k_scatter_K(Dims dm, int64_t nnzb, int64_t P, const int64_t* __restrict__ kc_ptr,
                            const int64_t* __restrict__ kc_src, LuDesc lud, const int* __restrict__ nbv,
                            const T* __restrict__ S, double* __restrict__ K, const int* __restrict__ fb_slot,
                            const double* __restrict__ fbS, const int* __restrict__ fb_count) {
  const int m2 = dm.m * dm.m;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nnzb * m2) return;
  const int64_t blk = idx / m2;
  const int i = (int)(idx % m2) / dm.m, k = (int)(idx % m2) % dm.m;
  double v = 0.0;
  if (lud.soff == nullptr) {
    const int64_t Nb = dm.Nb, nb2 = Nb * Nb, ld = dm.ld, n = dm.n;
    const int64_t row_off = dm.nu + (int64_t)i * Nb, col_off = dm.nu + (int64_t)k * Nb;
    const bool fb = fb_count != nullptr && *fb_count > 0;
    for (int64_t c = kc_ptr[blk]; c < kc_ptr[blk + 1]; ++c) {
      int64_t src = kc_src[c];
      int64_t e = src / nb2, s = (src / Nb) % Nb, t = src % Nb;
      const int sl = fb ? fb_slot[e] : -1;
      v += sl >= 0 ? fbS[((int64_t)sl * n + row_off + s) * ld + col_off + t]
                   : (double)S[(e * n + row_off + s) * ld + col_off + t];
    }
  } else {
    for (int64_t c = kc_ptr[blk]; c < kc_ptr[blk + 1]; ++c) {
      const int64_t src = kc_src[c];
      const int64_t e = src / (P * P), s = (src / P) % P, t = src % P;
      const int64_t nb = nbv[e], ld = lud.ld[e], nu = lud.nu[e];
      v += (double)S[lud.soff[e] + (nu + i * nb + s) * ld + nu + k * nb + t];
    }
  }
  K[idx] = v;
}

// Fault injection: u-row r of element e's bordered matrix (columns 0..n) set to zero,
// and its FP64 right-hand side entry on the mixed path.
template <class T>
__global__ void k_zero_row(T* __restrict__ row, int ncol, double* __restrict__ rhs_entry) {
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) row[c] = (T)0;
  if (threadIdx.x == 0 && rhs_entry) *rhs_entry = 0.0;
}

// Uniform meshes: one CTA per block row r of K.  The row's blocks accumulate in shared
// memory; each contribution (element e, slot s) reads the element's m trace rows of
// slot s (m x m Nb contiguous values per row: coalesced) and adds them to the blocks
// of the columns its slots map to (found by binary search in the row's sorted column
// list).  Contributions run in element order, as in k_scatter_K, so every block is the
// same sum in the same order; the row is then written out contiguously.
constexpr int SK_THREADS = 256;
template <class T>
__global__ void __launch_bounds__(SK_THREADS)
k_scatter_K_rows(Dims dm, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                 const int64_t* __restrict__ rc_ptr, const int64_t* __restrict__ rc_src,
                 const int64_t* __restrict__ etrace, const T* __restrict__ S, double* __restrict__ K,
                 const int* __restrict__ fb_slot, const double* __restrict__ fbS, const int* __restrict__ fb_count) {
  extern __shared__ double acc[];            // [blocks of the row][m][m]
  __shared__ int bmap[128];                  // slot t of the current element -> block of the row
  const int64_t r = blockIdx.x;
  const int tid = threadIdx.x;
  const int m = dm.m, m2 = m * m, Nb = dm.Nb, mNb = m * Nb;
  const int64_t b0 = row_ptr[r];
  const int nblk = (int)(row_ptr[r + 1] - b0);
  const int64_t n = dm.n, ld = dm.ld, nu = dm.nu;
  for (int i = tid; i < nblk * m2; i += SK_THREADS) acc[i] = 0.0;
  const bool fb = fb_count != nullptr && *fb_count > 0;
  for (int64_t c = rc_ptr[r]; c < rc_ptr[r + 1]; ++c) {
    const int64_t src = rc_src[c];
    const int64_t e = src / Nb;
    const int s = (int)(src % Nb);
    __syncthreads();                         // the previous contribution is done with bmap
    for (int t = tid; t < Nb; t += SK_THREADS) {
      const int32_t cc = (int32_t)etrace[e * Nb + t];
      int lo = 0, hi = nblk;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (col[b0 + mid] < cc) lo = mid + 1;
        else hi = mid;
      }
      bmap[t] = lo;
    }
    __syncthreads();
    const int sl = fb ? fb_slot[e] : -1;
    for (int idx = tid; idx < m * mNb; idx += SK_THREADS) {
      const int i = idx / mNb, kt = idx % mNb, k = kt / Nb, t = kt % Nb;
      const int64_t off = (nu + (int64_t)i * Nb + s) * ld + nu + kt;
      const double v = sl >= 0 ? fbS[(int64_t)sl * n * ld + off] : (double)S[e * n * ld + off];
      acc[bmap[t] * m2 + i * m + k] += v;
    }
  }
  __syncthreads();
  for (int i = tid; i < nblk * m2; i += SK_THREADS) K[b0 * m2 + i] = acc[i];
}

// Ragged form of k_scatter_R: contributions packed as e P + s, values located by src.
__global__ void k_scatter_R_ragged(int m, int64_t T, int64_t P, const int64_t* __restrict__ rc_ptr,
                                   const int64_t* __restrict__ rc_src, RaggedSrc rs,
                                   const double* __restrict__ src, double* __restrict__ R) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= T * m) return;
  const int64_t t = idx / m;
  const int i = (int)(idx % m);
  double v = 0.0;
  for (int64_t c = rc_ptr[t]; c < rc_ptr[t + 1]; ++c) {
    const int64_t es = rc_src[c];
    const int64_t e = es / P, s = es % P;
    v += src[rs.base[e] + s * rs.ss[e] + i * rs.cs[e]];
  }
  R[idx] = v;
}

// Nodal arrays between the user layout of a mesh with mixed orders (elements in user
// order, each its own number of nodes) and a child's [E][Np][w] layout.
__global__ void k_nodal_copy(int64_t E, int npw, int w, const int64_t* __restrict__ gnode,
                             const double* __restrict__ src, double* __restrict__ dst, bool to_child) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= E * npw) return;
  const int64_t e = idx / npw, r = idx % npw;
  const int64_t ui = gnode[e] * w + r;
  if (to_child) dst[idx] = src[ui];
  else dst[ui] = src[idx];
}

// One thread per (trace node, component): R[t][i] = sum over (e, s) of src(e, s, i).
__global__ void k_scatter_R(Dims dm, int64_t T, const int64_t* __restrict__ rc_ptr,
                            const int64_t* __restrict__ rc_src, const double* __restrict__ src,
                            int64_t es, int64_t ss, int64_t cs, double* __restrict__ R) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= T * dm.m) return;
  const int64_t t = idx / dm.m;
  const int i = (int)(idx % dm.m);
  double v = 0.0;
  for (int64_t c = rc_ptr[t]; c < rc_ptr[t + 1]; ++c) {
    int64_t es_ = rc_src[c];
    int64_t e = es_ / dm.Nb, s = es_ % dm.Nb;
    v += src[e * es + s * ss + i * cs];
  }
  R[idx] = v;
}

// One CTA per element.  rhs = (L^-1 P Ft) - (L^-1 P Bt) dU_e, du = U^-1 rhs,
// dq_kl = (q* - q) - G_l du_k + H_l dU_k.
constexpr int BS_THREADS = 256;
__global__ void __launch_bounds__(BS_THREADS)
k_backsub(Dims dm, Geo G, const int64_t* __restrict__ etrace, const double* __restrict__ S,
          const double* __restrict__ rhoq, const double* __restrict__ duhat,
          double* __restrict__ du, double* __restrict__ dq, TraceTab tt, const int64_t* __restrict__ elist) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = BS_THREADS / 32;
  // with an element list (FP64 fallback of the mixed path) CTA `slot` back-substitutes
  // element elist[slot] with the factors in matrix slot `slot`
  const int64_t slot = blockIdx.x;
  const int64_t e = elist ? elist[slot] : slot;
  if (e < 0) return;
  const int m = dm.m, d = dm.d, Np = dm.Np, NbT = dm.Nb, nu = dm.nu;
  const int Nb = tt.nb ? tt.nb[e] : NbT;      // this element's slots (mixed orders: ragged)
  const int nt = m * Nb;
  const int ld = tt.nb ? tt.ldv[e] : dm.ld;
  const double* A = S + (tt.nb ? tt.soff[e] : slot * (int64_t)dm.n * dm.ld);
  double* sU = sm;          // [nt]   dU_e, component-major (k Nb + t)
  double* y = sU + dm.nt;   // [nu]
  for (int idx = tid; idx < nt; idx += BS_THREADS) {
    int k = idx / Nb, t = idx % Nb;
    sU[idx] = duhat[etrace[e * NbT + t] * m + k];
  }
  __syncthreads();
  for (int r = warp; r < nu; r += nw) {
    const double* row = A + (int64_t)r * ld + nu;
    double s = 0.0;
    for (int c = lane; c < nt; c += 32) s = fma(row[c], sU[c], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[r] = row[nt] - s;
  }
  __syncthreads();
  for (int j = nu - 1; j >= 0; --j) {
    if (tid == 0) y[j] = y[j] / A[(int64_t)j * ld + j];
    __syncthreads();
    const double yj = y[j];
    for (int r = tid; r < j; r += BS_THREADS) y[r] = fma(-A[(int64_t)r * ld + j], yj, y[r]);
    __syncthreads();
  }
  for (int idx = tid; idx < Np * m; idx += BS_THREADS) {
    int b = idx / m, k = idx % m;
    du[e * Np * m + idx] = y[k * Np + b];
  }
  for (int idx = tid; idx < Np * m * d; idx += BS_THREADS) {
    int c = idx / (m * d), k = (idx / d) % m, l = idx % d;
    const double* gl = G.Gl + (((size_t)e * d + l) * Np + c) * Np;
    const double* hl = G.Hl + (((size_t)e * d + l) * Np + c) * NbT;
    double s = -rhoq[e * Np * m * d + idx];
    for (int b = 0; b < Np; ++b) s = fma(-gl[b], y[k * Np + b], s);
    for (int t = 0; t < Nb; ++t) s = fma(hl[t], sU[k * Nb + t], s);
    dq[e * Np * m * d + idx] = s;
  }
}

}  // namespace

cudaError_t launch_zero_row(iedg_mesh* M, cudaStream_t st) {
  const Dims& dm = M->dm;
  const int64_t e = M->fault.zero_row_elem;
  if (e < 0 || e >= M->E || M->fault.zero_row < 0 || M->fault.zero_row >= dm.nu) return cudaSuccess;
  const int64_t off = (e * dm.n + M->fault.zero_row) * (int64_t)dm.ld;
  if (M->precision == IEDG_PRECISION_FP64)
    k_zero_row<double><<<1, 128, 0, st>>>(M->S + off, dm.n + 1, nullptr);
  else
    k_zero_row<float><<<1, 128, 0, st>>>(M->S32 + off, dm.n + 1, M->rhs64 + e * dm.n + M->fault.zero_row);
  return cudaGetLastError();
}

cudaError_t launch_scatter_K(iedg_mesh* M, double* K, cudaStream_t st) {
  const int64_t total = M->nnzb * M->dm.m * M->dm.m;
  if (total == 0) return cudaSuccess;
  const size_t rsm = sizeof(double) * (size_t)M->max_row_blocks * M->dm.m * M->dm.m;
  if (M->lud.soff == nullptr && M->dm.Nb <= 128 && rsm <= 200 * 1024) {
    // uniform meshes: one CTA per block row, coalesced reads of the element rows
    cudaError_t err;
    if (M->precision == 0) {
      err = cudaFuncSetAttribute(k_scatter_K_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
      if (err != cudaSuccess) return err;
      k_scatter_K_rows<double><<<(unsigned)M->T, SK_THREADS, rsm, st>>>(M->dm, M->row_ptr, M->col, M->rc_ptr,
                                                                        M->rc_src, M->etrace, M->S, K, nullptr,
                                                                        nullptr, nullptr);
    } else {
      err = cudaFuncSetAttribute(k_scatter_K_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
      if (err != cudaSuccess) return err;
      k_scatter_K_rows<float><<<(unsigned)M->T, SK_THREADS, rsm, st>>>(M->dm, M->row_ptr, M->col, M->rc_ptr,
                                                                       M->rc_src, M->etrace, M->S32, K, M->fb_slot,
                                                                       M->fb_S, M->fb_S ? M->fb_count : nullptr);
    }
    return cudaGetLastError();
  }
  const int th = 256;
  const unsigned grid = (unsigned)((total + th - 1) / th);
  if (M->precision == 0)
    k_scatter_K<double><<<grid, th, 0, st>>>(M->dm, M->nnzb, M->nb_pack, M->kc_ptr, M->kc_src, M->lud, M->el_nb,
                                              M->S, K, nullptr, nullptr, nullptr);
  else
    k_scatter_K<float><<<grid, th, 0, st>>>(M->dm, M->nnzb, M->nb_pack, M->kc_ptr, M->kc_src, M->lud, M->el_nb,
                                             M->S32, K, M->fb_slot, M->fb_S, M->fb_S ? M->fb_count : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_scatter_R_ragged(iedg_mesh* M, const RaggedSrc& rs, const double* src, double* R,
                                    cudaStream_t st) {
  const int64_t total = M->T * M->dm.m;
  const int th = 256;
  k_scatter_R_ragged<<<(unsigned)((total + th - 1) / th), th, 0, st>>>(M->dm.m, M->T, M->nb_pack, M->rc_ptr,
                                                                        M->rc_src, rs, src, R);
  return cudaGetLastError();
}

cudaError_t launch_nodal_copy(iedg_mesh* C, int w, const double* src, double* dst, bool to_child,
                              cudaStream_t st) {
  const int64_t total = C->E * C->dm.Np * w;
  if (total == 0) return cudaSuccess;
  const int th = 256;
  k_nodal_copy<<<(unsigned)((total + th - 1) / th), th, 0, st>>>(C->E, C->dm.Np * w, w, C->gnode, src, dst,
                                                                  to_child);
  return cudaGetLastError();
}

cudaError_t launch_scatter_R(iedg_mesh* M, const double* src, int64_t es, int64_t ss, int64_t cs, double* R,
                             cudaStream_t st) {
  const int64_t total = M->T * M->dm.m;
  const int th = 256;
  k_scatter_R<<<(unsigned)((total + th - 1) / th), th, 0, st>>>(M->dm, M->T, M->rc_ptr, M->rc_src, src, es, ss,
                                                                  cs, R);
  return cudaGetLastError();
}

cudaError_t launch_backsub(iedg_mesh* M, const double* duhat, double* du, double* dq, cudaStream_t st) {
  const Dims& dm = M->dm;
  size_t smem = sizeof(double) * (size_t)(dm.nt + dm.nu);
  k_backsub<<<(unsigned)M->E, BS_THREADS, smem, st>>>(dm, M->geo, M->etrace, M->S, M->rhoq, duhat, du, dq,
                                                      M->tt, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_backsub_list(iedg_mesh* M, const double* S, const int64_t* elist, int64_t n_slots,
                                const double* duhat, double* du, double* dq, cudaStream_t st) {
  const Dims& dm = M->dm;
  size_t smem = sizeof(double) * (size_t)(dm.nt + dm.nu);
  k_backsub<<<(unsigned)n_slots, BS_THREADS, smem, st>>>(dm, M->geo, M->etrace, S, M->rhoq, duhat, du, dq, M->tt,
                                                         elist);
  return cudaGetLastError();
}

// The fault injection's zero row in the FP64 slot of its element, when it has one.
__global__ void k_zero_row_slot(int64_t e, int r, const int* __restrict__ slot_of, double* __restrict__ S,
                                int64_t slot_stride, int ld, int ncol) {
  const int sl = slot_of[e];
  if (sl < 0) return;
  double* row = S + sl * slot_stride + (int64_t)r * ld;
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) row[c] = 0.0;
}

cudaError_t launch_zero_row_fallback(iedg_mesh* M, cudaStream_t st) {
  const Dims& dm = M->dm;
  const int64_t e = M->fault.zero_row_elem;
  if (M->fb_S == nullptr || e < 0 || e >= M->E) return cudaSuccess;
  k_zero_row_slot<<<1, 128, 0, st>>>(e, M->fault.zero_row, M->fb_slot, M->fb_S, (int64_t)dm.n * dm.ld, dm.ld,
                                     dm.n + 1);
  return cudaGetLastError();
}

}  // namespace iedg
