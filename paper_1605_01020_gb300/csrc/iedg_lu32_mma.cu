// FP32 partial LU of the mixed path (static condensation, Eq. LS) with every trailing
// update on the 5th-generation tensor cores.
//
// Same algorithm, pivot rule and stored factors as the FFMA form (k_lu32): panels of
// 32 columns, pivots searched among the u-rows only, the panel's interchanges applied
// to the panel and to the columns right of it (the L columns of earlier panels stay
// where they were), L and U kept in place for the refinement solves, K_e | R_e left in
// the trailing block.  What changes is where the work runs:
//
//   panel      the 32 panel columns live in shared memory in the tcgen05 K-major
//              operand layout (8-row x 16-byte core matrices).  They are factored in
//              groups of 4 columns: each thread holds the group's 4 values of its rows
//              in registers, so the pivot search, the row exchange and the rank-1
//              updates inside the group touch no shared memory; after the group its
//              U rows are finished (a 4-row triangular solve) and the rest of the panel
//              gets one rank-4 update.
//   U12        the panel's interchanges and L11^-1 on the columns right of the panel,
//              one column per thread (as in k_lu32).
//   trailing   A22 -= L21 U12 is a GEMM with K = 32 per panel: 128-row tiles of L21
//              (the panel buffer itself, high parts; low parts staged per row tile),
//              64-column tiles of U12 (staged from global memory, high and low parts),
//              three TF32 products per K step ("3xTF32": hi hi + hi lo + lo hi, FP32
//              accuracy), accumulated in tensor memory; the epilogue subtracts the
//              product from the trailing block in global memory.  Two accumulators:
//              the MMAs of one tile run while the epilogue of the previous tile reads
//              its accumulator and streams its part of the trailing block.
//
// TF32 splitting: x = hi + lo with hi = x with the low 13 mantissa bits cleared
// (exactly representable in TF32) and lo = x - hi exact in FP32; the products drop
// lo lo (below 2^-22 of |x y|).  The high parts are stored with the bits cleared, so
// nothing depends on how the tensor core treats the low bits of its inputs.
//
// Waits on the MMA completion barriers are bounded; a CTA whose wait gives up flags
// its element and every element it still takes from the queue IEDG_ELEM_TIMEOUT,
// waits (bounded) for its MMAs in flight and frees its tensor memory.
#include "iedg_internal.cuh"
#include "iedg_lu_common.cuh"
#include "iedg_tc.cuh"

namespace iedg {
namespace {

constexpr int MM_THREADS = 256;
constexpr int MM_NB = 32;                 // panel width = K of one trailing update
constexpr int MM_MAX_N = 6 * MM_THREADS;  // panel rows per thread (RPT) <= 6
constexpr int MM_TM = 128, MM_TN = 64;    // output tile of one MMA group
constexpr int MM_ALO_BYTES = MM_TM * MM_NB * 4;     // low parts of one row tile of L21
constexpr int MM_B_BYTES = MM_TN * MM_NB * 4;       // one part (hi or lo) of a U12 tile
constexpr int MM_TMEM_COLS = 2 * MM_TN;             // two accumulators

// Element (r, k) of a panel-layout buffer (rows x 32, core matrices, SBO 1024, LBO 128).
__device__ __forceinline__ float* pel(unsigned char* base, int r, int k) {
  return reinterpret_cast<float*>(base + tc::core_off32(r, k));
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

struct MmBufs {
  unsigned char* P;     // panel [n][32]
  unsigned char* Alo;   // low parts of one 128-row tile of L21
  unsigned char* Bhi;   // U12 tile, 64 x 32, high parts
  unsigned char* Blo;   //                     low parts
};

// Bytes of the panel buffer for an n-row element, padded so that the last row tile's
// MMA (which reads 128 rows from an 8-row boundary) stays inside the CTA's allocation:
// the rows past the element are followed by the staging buffers.
__host__ __device__ inline size_t mm_panel_bytes(int n) { return (size_t)((n + 7) / 8) * 8 * MM_NB * 4; }

// Panel factorisation of columns kb .. kb+nb-1 over rows kb .. n-1 (local rows 0..rows-1).
// Returns through perm / piv / pivots as k_lu32 does.
template <int RPT>
__device__ __forceinline__ void mm_panel(unsigned char* P, int rows, int prow, int nb, int kb, int* piv, int* perm,
                                         int* pivots, int64_t poff, float* xchg, float* rv, int* ri, int& sing,
                                         int& nonfin) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j0 = 0; j0 < nb; j0 += 4) {
    // the group's values of this thread's rows (rows above j0 are finished U rows)
    float v[RPT][4];
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      const int i = tid + s * MM_THREADS;
      if (i >= j0 && i < rows) {
        const float4 t = *reinterpret_cast<const float4*>(pel(P, i, j0));
        v[s][0] = t.x; v[s][1] = t.y; v[s][2] = t.z; v[s][3] = t.w;
      } else {
        v[s][0] = v[s][1] = v[s][2] = v[s][3] = 0.f;
      }
    }
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int j = j0 + jj;
      if (j >= nb) break;
      // pivot: largest |a| among the u-rows j .. prow-1, lowest row on ties
      float best = -1.f;
      int bi = j;
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        const int i = tid + s * MM_THREADS;
        if (i >= j && i < prow) {
          const float a = fabsf(v[s][jj]);
          nonfin |= !(a <= 3.402823466e38f);
          if (a > best) { best = a; bi = i; }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
      __syncthreads();
      float bv = rv[0];
      int pr = ri[0];
      for (int w = 1; w < MM_THREADS / 32; ++w)
        if (rv[w] > bv || (rv[w] == bv && ri[w] < pr)) { bv = rv[w]; pr = ri[w]; }
      if (!(bv > 0.f)) pr = j;
      // rows pr and j trade places: their group values go through xchg
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        const int i = tid + s * MM_THREADS;
        if (i == pr) { xchg[0] = v[s][0]; xchg[1] = v[s][1]; xchg[2] = v[s][2]; xchg[3] = v[s][3]; }
        if (i == j) { xchg[4] = v[s][0]; xchg[5] = v[s][1]; xchg[6] = v[s][2]; xchg[7] = v[s][3]; }
      }
      if (tid == 0) {
        if (!(bv > 0.f)) sing = 1;
        piv[j] = pr;
        pivots[poff + kb + j] = kb + pr;
        if (pr != j) { const int t = perm[j]; perm[j] = perm[pr]; perm[pr] = t; }
      }
      __syncthreads();
      const float u0 = xchg[0], u1 = xchg[1], u2 = xchg[2], u3 = xchg[3];
      const float uj[4] = {u0, u1, u2, u3};
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        const int i = tid + s * MM_THREADS;
        if (i == j) { v[s][0] = u0; v[s][1] = u1; v[s][2] = u2; v[s][3] = u3; }
        else if (i == pr) { v[s][0] = xchg[4]; v[s][1] = xchg[5]; v[s][2] = xchg[6]; v[s][3] = xchg[7]; }
      }
      // the other 28 columns of the two rows (the L part of earlier groups and the
      // columns not reached yet) are swapped in shared memory, one column per thread
      if (pr != j && tid < MM_NB && (tid < j0 || tid >= j0 + 4)) {
        float* a = pel(P, j, tid);
        float* b = pel(P, pr, tid);
        const float t = *a;
        *a = *b;
        *b = t;
      }
      const float inv = uj[jj] != 0.f ? 1.f / uj[jj] : 0.f;
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        const int i = tid + s * MM_THREADS;
        if (i > j && i < rows) {
          const float l = v[s][jj] * inv;
          v[s][jj] = l;
#pragma unroll
          for (int c = jj + 1; c < 4; ++c) v[s][c] = fmaf(-l, uj[c], v[s][c]);
        }
      }
    }
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      const int i = tid + s * MM_THREADS;
      if (i >= j0 && i < rows)
        *reinterpret_cast<float4*>(pel(P, i, j0)) = make_float4(v[s][0], v[s][1], v[s][2], v[s][3]);
    }
    __syncthreads();
    if (j0 + 4 >= MM_NB) break;
    // the group's U rows on the columns right of the group (4-row triangular solve)
    if (tid < MM_NB - j0 - 4) {
      const int c = j0 + 4 + tid;
      float uc[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float x = *pel(P, j0 + k, c);
#pragma unroll
        for (int l = 0; l < k; ++l) x = fmaf(-*pel(P, j0 + k, j0 + l), uc[l], x);
        uc[k] = x;
        if (j0 + k < nb) *pel(P, j0 + k, c) = x;
      }
    }
    __syncthreads();
    // rank-4 update of the rows below the group on the columns right of it
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      const int i = tid + s * MM_THREADS;
      if (i >= j0 + 4 && i < rows) {
        for (int c4 = (j0 + 4) >> 2; c4 < MM_NB / 4; ++c4) {
          float4 x = *reinterpret_cast<const float4*>(pel(P, i, 4 * c4));
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (j0 + k >= nb) break;
            const float4 u = *reinterpret_cast<const float4*>(pel(P, j0 + k, 4 * c4));
            const float l = v[s][k];
            x.x = fmaf(-l, u.x, x.x); x.y = fmaf(-l, u.y, x.y); x.z = fmaf(-l, u.z, x.z); x.w = fmaf(-l, u.w, x.w);
          }
          *reinterpret_cast<float4*>(pel(P, i, 4 * c4)) = x;
        }
      }
    }
    __syncthreads();
  }
}

// One tile of U12 (K rows kb.., columns c0 .. c0+63) as 8 values per thread, read
// from global memory ahead of its staging.
__device__ __forceinline__ void mm_load_b(const float* __restrict__ A, int ld, int kb, int nb, int c0, int ncol,
                                          float (&bv)[8]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int idx = threadIdx.x + q * MM_THREADS, k = idx >> 6, c = c0 + (idx & 63);
    bv[q] = (k < nb && c < ncol) ? __ldcg(A + (int64_t)(kb + k) * ld + c) : 0.f;
  }
}

__device__ __forceinline__ void mm_stage_b(const MmBufs& b, const float (&bv)[8]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int idx = threadIdx.x + q * MM_THREADS, k = idx >> 6, nn = idx & 63;
    const float hi = tf32_hi(bv[q]);
    *pel(b.Bhi, nn, k) = hi;
    *pel(b.Blo, nn, k) = bv[q] - hi;
  }
}

// Low parts of panel rows r .. r+127 into Alo; the panel rows keep their high parts.
// Rows at or past `rows` (the last tile's overhang, read by the MMA but never stored
// back) get zero low parts and leave the memory behind the panel untouched.
__device__ __forceinline__ void mm_stage_a(const MmBufs& b, int r, int rows) {
#pragma unroll
  for (int q = 0; q < (MM_TM * MM_NB / 4) / MM_THREADS; ++q) {
    const int idx = threadIdx.x + q * MM_THREADS, rr = idx >> 3, k = (idx & 7) * 4;
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r + rr < rows) {
      float4* src = reinterpret_cast<float4*>(pel(b.P, r + rr, k));
      const float4 x = *src;
      float4 h;
      h.x = tf32_hi(x.x); h.y = tf32_hi(x.y); h.z = tf32_hi(x.z); h.w = tf32_hi(x.w);
      lo = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      *src = h;
    }
    *reinterpret_cast<float4*>(pel(b.Alo, rr, k)) = lo;
  }
}

__device__ __forceinline__ void mm_issue(uint32_t tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo) {
  constexpr uint32_t IDESC = tc::idesc_tf32(MM_TM, MM_TN);
  // one instruction covers K = 8: two core matrices along K (LBO 128, SBO 1024)
#pragma unroll
  for (int st = 0; st < MM_NB / 8; ++st) {
    const uint32_t ko = st * 256;
    tc::mma_tf32(tmem, tc::desc_kmajor(a_hi + ko, 128, 1024), tc::desc_kmajor(b_hi + ko, 128, 1024), IDESC,
                 st == 0 ? 0u : 1u);
    tc::mma_tf32(tmem, tc::desc_kmajor(a_hi + ko, 128, 1024), tc::desc_kmajor(b_lo + ko, 128, 1024), IDESC, 1u);
    tc::mma_tf32(tmem, tc::desc_kmajor(a_lo + ko, 128, 1024), tc::desc_kmajor(b_hi + ko, 128, 1024), IDESC, 1u);
  }
}

// A[r][c] -= acc[r][c] for the tile at (rt, ct): warp (q, h) owns TMEM lanes 32 q ..
// 32 q + 31 (rows rt + 32 q + lane) and columns 32 h .. 32 h + 31.  Rows below r_lo
// (inside an 8-row group above the trailing block) and past n, columns past ncol are
// left alone.  The subtraction is a reduction performed in L2 (red.global.add of
// -acc, four values per instruction on 16-byte boundaries): the SM never waits for
// the trailing block's values, and each entry receives exactly one update per panel,
// so the result does not depend on timing.
__device__ __forceinline__ void mm_epilogue(float* __restrict__ A, int ld, int n, int ncol, int r_lo, int rt,
                                            int ct, uint32_t tacc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, q = warp & 3, h = warp >> 2;
  const int row = rt + 32 * q + lane, c0 = ct + 32 * h;
  const bool live = row >= r_lo && row < n && c0 < ncol;
  float* dst = A + (int64_t)row * ld + c0;
  const bool vec = live && ((c0 & 3) == 0) && c0 + 32 <= ncol;
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) {
    float acc[16];
    tc::tmem_ld16(tacc + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * h + 16 * hf), acc);
    if (vec) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + 16 * hf + 4 * j),
                     "f"(-acc[4 * j]), "f"(-acc[4 * j + 1]), "f"(-acc[4 * j + 2]), "f"(-acc[4 * j + 3])
                     : "memory");
    } else if (live) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (c0 + 16 * hf + j < ncol) atomicAdd(dst + 16 * hf + j, -acc[j]);
    }
  }
}

// Bounded wait on accumulator b's barrier by every thread, outcome made uniform.
__device__ __forceinline__ bool mm_wait(TcState& t, int b) {
  const bool ok = __syncthreads_and(tc::mbar_wait(t.mbar + b, t.phase[b], t.limit));
  if (ok) { t.phase[b] ^= 1u; t.pending[b] = 0; }
  else t.failed = 1;
  return ok;
}

// Trailing update A[r0:n, r0:ncol] -= L21 U12 of the panel at kb (nb columns): row tiles
// of 128 from the 8-row boundary at or above r0 (outer), column tiles of 64 (inner).
__device__ void mm_trailing(float* __restrict__ A, int ld, int n, int kb, int nb, const MmBufs& b, TcState& t) {
  const int tid = threadIdx.x;
  const int ncol = n + 1, r0 = kb + nb;
  const int rs = nb & ~7;                               // first row tile, local to the panel
  const int n_mt = (n - kb - rs + MM_TM - 1) / MM_TM;
  const int n_nt = (ncol - r0 + MM_TN - 1) / MM_TN;
  const int T = n_mt * n_nt;
  const uint32_t aP = tc::smem_u32(b.P), aLo = tc::smem_u32(b.Alo), bHi = tc::smem_u32(b.Bhi),
                 bLo = tc::smem_u32(b.Blo);
  float bv[8];
  mm_load_b(A, ld, kb, nb, r0, ncol, bv);
  for (int it = 0; it <= T && !t.failed; ++it) {
    if (it < T) {
      const int mt = it / n_nt, nt = it % n_nt;
      // the MMAs of the previous tile read Alo, the B tile and (last row tile) the rows
      // past the panel; they finish before anything is restaged
      if (it >= 1 && !mm_wait(t, (it - 1) & 1)) break;
      if (nt == 0) mm_stage_a(b, rs + mt * MM_TM, n - kb);
      mm_stage_b(b, bv);
      tc::fence_proxy_async();
      __syncthreads();
      tc::fence_after_sync();
      if (tid == 0) {
        mm_issue(t.tmem + (uint32_t)((it & 1) * MM_TN), aP + (uint32_t)((rs + mt * MM_TM) >> 3) * 1024u, aLo, bHi,
                 bLo);
        tc::mma_commit(t.mbar + (it & 1));
      }
      t.pending[it & 1] = 1;
      // the next tile's U12 values, read while this tile's MMAs and the previous
      // tile's epilogue run
      if (it + 1 < T) mm_load_b(A, ld, kb, nb, r0 + ((it + 1) % n_nt) * MM_TN, ncol, bv);
    } else if (!mm_wait(t, (it - 1) & 1)) {
      break;
    }
    if (it >= 1) {
      const int pm = (it - 1) / n_nt, pn = (it - 1) % n_nt;
      tc::fence_after_sync();
      mm_epilogue(A, ld, n, ncol, r0, kb + rs + pm * MM_TM, r0 + pn * MM_TN,
                  t.tmem + (uint32_t)(((it - 1) & 1) * MM_TN));
      tc::fence_before_sync();
    }
  }
  __syncthreads();
}

template <int RPT>
__device__ void mm_element(const LuElem& el, float* __restrict__ S, int8_t* __restrict__ status,
                           int* __restrict__ pivots, int64_t e, TcState& t) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ int piv[MM_NB];
  __shared__ int perm[LU_MAX_NU];
  __shared__ float rv[MM_THREADS / 32];
  __shared__ int ri[MM_THREADS / 32];
  __shared__ float xchg[8];
  __shared__ int sing;
  const int tid = threadIdx.x;
  const int n = el.n, nu = el.nu, ld = el.ld, ncol = n + 1;
  float* A = S + el.off;
  MmBufs b;
  b.P = smraw;
  b.Alo = smraw + mm_panel_bytes(n);
  b.Bhi = b.Alo + MM_ALO_BYTES;
  b.Blo = b.Bhi + MM_B_BYTES;
  int nonfin = 0;
  if (tid == 0) sing = 0;
  for (int kb = 0; kb < nu && !t.failed; kb += MM_NB) {
    const int nb = min(MM_NB, nu - kb), rows = n - kb, prow = nu - kb;
    // panel load (columns past nb are zero), eight independent loads per thread in flight
    for (int base = 0; base < rows * 8; base += 8 * MM_THREADS) {
      float4 x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * MM_THREADS + tid, r = idx >> 3, k = (idx & 7) * 4;
        x[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < rows * 8) {
          const float* src = A + (int64_t)(kb + r) * ld + kb + k;
          if (k + 4 <= nb) {
            x[u] = __ldcg(reinterpret_cast<const float4*>(src));
          } else {
            x[u].x = k < nb ? __ldcg(src) : 0.f;
            x[u].y = k + 1 < nb ? __ldcg(src + 1) : 0.f;
            x[u].z = k + 2 < nb ? __ldcg(src + 2) : 0.f;
            x[u].w = k + 3 < nb ? __ldcg(src + 3) : 0.f;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * MM_THREADS + tid;
        if (idx < rows * 8) *reinterpret_cast<float4*>(pel(b.P, idx >> 3, (idx & 7) * 4)) = x[u];
      }
    }
    for (int r = tid; r < prow; r += MM_THREADS) perm[r] = r;
    __syncthreads();
    mm_panel<RPT>(b.P, rows, prow, nb, kb, piv, perm, pivots, el.poff, xchg, rv, ri, sing, nonfin);
    // the full panel (U11, L11, L21) back to the element matrix for the refinement solves
    for (int idx = tid; idx < rows * 8; idx += MM_THREADS) {
      const int r = idx >> 3, k = (idx & 7) * 4;
      if (k >= nb) continue;
      const float4 x = *reinterpret_cast<const float4*>(pel(b.P, r, k));
      float* dst = A + (int64_t)(kb + r) * ld + kb + k;
      if (k + 4 <= nb) {
        *reinterpret_cast<float4*>(dst) = x;
      } else {
        dst[0] = x.x;
        if (k + 1 < nb) dst[1] = x.y;
        if (k + 2 < nb) dst[2] = x.z;
      }
    }
    // columns right of the panel: the panel's interchanges, then U12 = L11^-1 A12 (as in
    // k_lu32: each column gathers its new top rows, moves the displaced rows in groups
    // of 8, then solves with L11)
    for (int c = kb + nb + tid; c < ncol; c += MM_THREADS) {
      float x[MM_NB];
#pragma unroll
      for (int j = 0; j < MM_NB; ++j) {
        if (j >= nb) break;
        x[j] = __ldcg(A + (int64_t)(kb + perm[j]) * ld + c);
      }
#pragma unroll
      for (int j0 = 0; j0 < MM_NB; j0 += 8) {
        float y[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int r = j0 + j < nb ? piv[j0 + j] : 0;
          y[j] = (j0 + j < nb && r >= nb && perm[r] != r) ? __ldcg(A + (int64_t)(kb + perm[r]) * ld + c) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int r = j0 + j < nb ? piv[j0 + j] : 0;
          if (j0 + j < nb && r >= nb && perm[r] != r) A[(int64_t)(kb + r) * ld + c] = y[j];
        }
      }
#pragma unroll
      for (int j = 0; j < MM_NB; ++j) {
        if (j >= nb) break;
        float s = x[j];
#pragma unroll
        for (int jj = 0; jj < MM_NB; ++jj) {
          if (jj >= j) break;
          s = fmaf(-*pel(b.P, j, jj), x[jj], s);
        }
        x[j] = s;
        A[(int64_t)(kb + j) * ld + c] = s;
      }
    }
    __syncthreads();
    if (kb + nb < n) {
      mm_trailing(A, ld, n, kb, nb, b, t);
      // the trailing block's reductions are performed (gpu scope) before any thread of
      // the CTA reads it again; those reads go to L2 (ld.global.cg), past any line an
      // earlier load left in L1
      __threadfence();
      __syncthreads();
    }
  }
  __syncthreads();
  int bad = 0;
  for (int idx = tid; idx < (n - nu) * (ncol - nu); idx += MM_THREADS) {
    const int r = nu + idx / (ncol - nu), c = nu + idx % (ncol - nu);
    if (!isfinite(__ldcg(A + (int64_t)r * ld + c))) bad = 1;
  }
  bad = __syncthreads_or(bad);
  nonfin = __syncthreads_or(nonfin);
  if (tid == 0) {
    if (t.failed) status[e] = IEDG_ELEM_TIMEOUT;
    else status[e] = nonfin ? IEDG_ELEM_NONFINITE
                            : (sing ? IEDG_ELEM_SINGULAR : (bad ? IEDG_ELEM_NONFINITE : IEDG_ELEM_OK));
  }
  __syncthreads();
}

template <int RPT>
__global__ void __launch_bounds__(MM_THREADS, RPT <= 3 ? 2 : 1)
k_lu32_mma(Dims dm, LuDesc lud, float* __restrict__ S, int8_t* __restrict__ status, int* __restrict__ pivots,
           int64_t* queue, int64_t E, int* err, int wait_limit) {
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar[2];
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, MM_TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  TcState t;
  t.tmem = tmem_base;
  t.mbar = mbar;
  t.phase[0] = t.phase[1] = 0;
  t.pending[0] = t.pending[1] = 0;
  t.failed = 0;
  t.limit = wait_limit;
  int64_t e;
  int64_t it = 0;
  for (; next_element(queue, E, it, lud.order, &e); ++it) {
    mm_element<RPT>(lu_elem(dm, lud, e), S, status, pivots, e, t);
    if (t.failed) {
      if (tid == 0) atomicOr(err, 1);
      tc_drain(t);
      ++it;
      break;
    }
  }
  if (t.failed)
    for (; next_element(queue, E, it, lud.order, &e); ++it)
      if (tid == 0) status[e] = IEDG_ELEM_TIMEOUT;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem_base, MM_TMEM_COLS);
}

}  // namespace

size_t lu32_mma_smem(int n_max) {
  return mm_panel_bytes(n_max) + MM_ALO_BYTES + 2 * MM_B_BYTES;
}

template <int RPT>
static cudaError_t lu32_mma(iedg_mesh* M, int n_max, cudaStream_t st) {
  const size_t smem = lu32_mma_smem(n_max);
  cudaError_t err = cudaFuncSetAttribute(k_lu32_mma<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  unsigned grid = (unsigned)M->E;
  int64_t* queue = nullptr;
  if (M->sched.lu_persistent) {
    // at most 4 resident CTAs: each holds 128 of the SM's 512 TMEM columns
    err = persistent_grid(k_lu32_mma<RPT>, smem, M->E, &grid, 4, MM_THREADS);
    if (err == cudaSuccess) err = cudaMemsetAsync(M->queue, 0, sizeof(int64_t), st);
    if (err != cudaSuccess) return err;
    queue = M->queue;
  }
  k_lu32_mma<RPT><<<grid, MM_THREADS, smem, st>>>(M->dm, M->lud, M->S32, M->status, M->piv, queue, M->E,
                                                  M->dev_flag, tc_wait_limit(M));
  return cudaGetLastError();
}

cudaError_t launch_lu32_mma(iedg_mesh* M, int n_max, cudaStream_t st) {
  if (n_max > MM_MAX_N) return cudaErrorInvalidValue;
  return n_max <= 3 * MM_THREADS ? lu32_mma<3>(M, n_max, st) : lu32_mma<6>(M, n_max, st);
}

}  // namespace iedg
