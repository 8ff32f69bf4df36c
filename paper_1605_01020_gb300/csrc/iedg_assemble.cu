// Element block assembly with the q-elimination folded in at the quadrature points,
// and the partial LU of the bordered element matrix (static condensation, Eq. LS).
//
// Bordered element matrix (rows x cols = n x (n+1), n = m Np + m Nb):
//     [ At  Bt  Ft ]     rows i Np + a      (u-equation i, node a)
//     [ Ct  Dt  Gt ]     rows nu + i Nb + s (trace equation i, slot s)
// columns k Np + b (u unknown k, node b), nu + k Nb + t (trace unknown k, slot t), n.
// A_qq = M (x) I (Eq. IEDG a) lets q be eliminated exactly:
//   dq_kl = M^-1 F_q,kl - G_l du_k + H_l dU_k,
// so with the lifted operators Gl(g) = Phi G_l, Hl(g) = Phi H_l at the points,
//   At_ik[a][b] = alpha delta_ik M_ab
//              + sum_{g,r} Dxi_r[g][a] (cu_ikr(g) Phi[g][b] - sum_l cq_iklr(g) Gl_l(g)[b])
//              + sum_fp PhiF[fp][a] (lamw delta_ik PhiF[fp][b] - sum_l fq_ikl(fp) GlF_l(fp)[b])
//   Bt_ik[a][t] = sum_{g,r} Dxi_r[g][a] sum_l cq_iklr(g) Hl_l(g)[t]
//              + sum_fp PhiF[fp][a] (fuh_ik(fp) mu_t(fp) + sum_l fq_ikl(fp) HlF_l(fp)[t])
// and the trace rows Ct, Dt equal the face parts of the u-rows of the boundary nodes
// (mu_s = phi_bnode[s] on every face), which is how they are formed here.
// The right-hand-side column is written by the point kernel: Ft = -R_u(u, q*),
// Gt = -R_FL,e(u, q*) (exact because the fluxes are affine in q).
#include <cuda_bf16.h>

#include "iedg_internal.cuh"
#include "iedg_lu_common.cuh"
#include "iedg_tc.cuh"

namespace iedg {
namespace {

constexpr int AS_THREADS = 256;
constexpr int TM = 4, TN = 8;       // register tile of the volume contraction
constexpr int GC = 8;               // volume points per K-chunk

struct AsmCfg {
  int rows_pad;   // Np rounded up to TM
  int rg;         // row groups
  int CW;         // columns per CTA (multiple of TN)
  int cg;         // column groups
  int nsplit;     // CTAs per (element, i, k)
  int KC;         // K-chunk rows = GC d
};

AsmCfg asm_cfg(const Dims& dm) {
  AsmCfg c;
  c.rows_pad = idiv_up(dm.Np, TM) * TM;
  c.rg = c.rows_pad / TM;
  int max_cg = AS_THREADS / c.rg;
  int need = idiv_up(dm.Np + dm.Nb, TN);
  c.nsplit = idiv_up(need, max_cg);
  c.cg = idiv_up(need, c.nsplit);
  c.CW = c.cg * TN;
  c.KC = GC * dm.d;
  return c;
}

// T = double: FP64 path.  T = float: mixed path (FP32 element matrix; the FP64
// right-hand sides are copied into column n by one CTA per element).
// Meshes with mixed orders (tt.nb set): per-element slot count, offset and leading
// dimension; the trace basis at the face points comes from the element's table, and
// the trace rows are accumulated separately from the face parts of the u-rows.
template <class T, bool LIST = false>
__global__ void __launch_bounds__(AS_THREADS)
k_assemble(Dims dm, Phys ph, AsmCfg cf, RefTables ref, AsmTab<T> tb, T* __restrict__ S,
           const double* __restrict__ rhs64, TraceTab tt, int NbU, const int64_t* __restrict__ elist) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int tid = threadIdx.x;
  const int m2 = dm.m * dm.m;
  // the m^2 CTAs of an element are adjacent; with an element list (FP64 fallback of the
  // mixed path) CTA group `slot` assembles element elist[slot] into matrix slot `slot`
  const int64_t slot = blockIdx.x / m2;
  int64_t e = slot;
  if constexpr (LIST) {
    e = elist[slot];
    if (e < 0) return;
  }
  const int pair = blockIdx.x % m2, i = pair / dm.m, k = pair % dm.m;
  const int c0 = blockIdx.y * cf.CW;
  const int d = dm.d, Np = dm.Np, Nq = dm.Nq, Nfp = dm.Nfp, Nfq = dm.Nfq, Nfn = dm.Nfn;
  const bool mix = tt.nb != nullptr;
  const int NbT = dm.Nb;                            // slot stride of the lifting tables
  const int Nb = mix ? tt.nb[e] : dm.Nb;            // trace slots of this element
  const int ncol = Np + Nb;
  const int KC = cf.KC, CW = cf.CW, RP = cf.rows_pad;
  T* sA = sm;                           // [KC][RP]   Dxi_r[g][a]
  T* sB = sA + KC * RP;                 // [KC][CW]   W[(g, r)][col]
  T* facc = sB + KC * CW;               // [NbU][CW]  face parts of the boundary rows
  T* sV = facc + NbU * CW;              // [Nfq][CW]  face right operand
  T* tacc = mix ? sV + Nfq * CW : facc; // [Nb][CW]   trace rows (mixed orders), else = facc
  const T* mutab = nullptr;
  if (mix) {
    if constexpr (sizeof(T) == 8) mutab = reinterpret_cast<const T*>(tt.muf);
    else mutab = reinterpret_cast<const T*>(tt.muf32);
    mutab += (size_t)e * dm.nf * Nfq * tt.NFS;
  }
  const size_t jvs = (size_t)(1 + d) * d * Nq;
  const T* jv = tb.Jv + ((size_t)e * dm.m * dm.m + pair) * jvs;
  const size_t jfs = (size_t)(1 + d) * Nfp;
  const T* jf = tb.Jf + ((size_t)e * dm.m * dm.m + pair) * jfs;
  const T* GlV = tb.GlV + (size_t)e * d * Nq * Np;
  const T* HlV = tb.HlV + (size_t)e * d * Nq * NbT;
  const T* GlF = tb.GlF + (size_t)e * d * Nfp * Np;
  const T* HlF = tb.HlF + (size_t)e * d * Nfp * NbT;

  const int trow = tid / cf.cg, tcol = tid % cf.cg;
  const bool gemm_thread = trow < cf.rg;
  T acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = (T)0;

  // ---- volume contraction, K = Nq d in chunks of GC points
  for (int g0 = 0; g0 < Nq; g0 += GC) {
    for (int idx = tid; idx < KC * RP; idx += AS_THREADS) {
      int kc = idx / RP, a = idx % RP;
      int g = g0 + kc / d, r = kc % d;
      sA[idx] = (g < Nq && a < Np) ? tb.Dxi[((size_t)r * Nq + g) * Np + a] : (T)0;
    }
    for (int idx = tid; idx < KC * CW; idx += AS_THREADS) {
      int kc = idx / CW, col = c0 + idx % CW;
      int g = g0 + kc / d, r = kc % d;
      T w = 0;
      if (g < Nq && col < ncol) {
        if (col < Np) {
          w = jv[(size_t)r * Nq + g] * tb.Phi[(size_t)g * Np + col];
          for (int l = 0; l < d; ++l)
            w -= jv[(size_t)(d + l * d + r) * Nq + g] * GlV[((size_t)l * Nq + g) * Np + col];
        } else {
          for (int l = 0; l < d; ++l)
            w += jv[(size_t)(d + l * d + r) * Nq + g] * HlV[((size_t)l * Nq + g) * NbT + (col - Np)];
        }
      }
      sB[idx] = w;
    }
    __syncthreads();
    if (gemm_thread) {
      for (int kc = 0; kc < KC; ++kc) {
        T av[TM], bv[TN];
#pragma unroll
        for (int a = 0; a < TM; ++a) av[a] = sA[kc * RP + trow * TM + a];
#pragma unroll
        for (int b = 0; b < TN; ++b) bv[b] = sB[kc * CW + tcol * TN + b];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TN; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
      }
    }
    __syncthreads();
  }

  // ---- face parts, accumulated per trace slot
  for (int idx = tid; idx < NbU * CW; idx += AS_THREADS) facc[idx] = (T)0;
  if (mix)
    for (int idx = tid; idx < Nb * CW; idx += AS_THREADS) tacc[idx] = (T)0;
  const T lamsel = (i == k) ? (T)1 : (T)0;
  for (int f = 0; f < dm.nf; ++f) {
    __syncthreads();
    for (int idx = tid; idx < Nfq * CW; idx += AS_THREADS) {
      int gf = idx / CW, col = c0 + idx % CW;
      int fp = f * Nfq + gf;
      T v = 0;
      if (col < Np) {
        // dfhat/du: lambda I (Lax-Friedrichs) or the pair's entry of S (Roe-type)
        const T su = tb.Su ? tb.Su[((size_t)e * dm.m * dm.m + pair) * Nfp + fp] : lamsel * tb.lamw[e * Nfp + fp];
        v = su * tb.PhiF[(size_t)fp * Np + col];
        for (int l = 0; l < d; ++l) v -= jf[(size_t)(1 + l) * Nfp + fp] * GlF[((size_t)l * Nfp + fp) * Np + col];
      } else if (col < ncol) {
        int t = col - Np;
        T mu = 0;
        if (mix) {
          const int* fl = tt.sfl + ((size_t)e * NbT + t) * 3;
          for (int q = 0; q < 3; ++q) {
            const int code = fl[q];
            if (code >= 0 && code / tt.NFS == f) mu = mutab[((size_t)f * Nfq + gf) * tt.NFS + code % tt.NFS];
          }
        } else {
          mu = tb.PhiF[(size_t)fp * Np + ref.bnode[t]];
        }
        v = jf[fp] * mu;
        for (int l = 0; l < d; ++l) v += jf[(size_t)(1 + l) * Nfp + fp] * HlF[((size_t)l * Nfp + fp) * NbT + t];
      }
      sV[idx] = v;
    }
    __syncthreads();
    for (int idx = tid; idx < Nfn * CW; idx += AS_THREADS) {
      int tn = idx / CW, cc = idx % CW;
      int a = ref.fnode[f * Nfn + tn];
      T s = 0;
      for (int gf = 0; gf < Nfq; ++gf) s += tb.PhiF[(size_t)(f * Nfq + gf) * Np + a] * sV[gf * CW + cc];
      facc[ref.slot[a] * CW + cc] += s;
    }
    if (mix) {
      // domain-boundary face: the trace rows take the boundary flux, so the right
      // operand is rebuilt from its derivatives
      if (tt.fkind && tt.fkind[e * dm.nf + f] != kFaceInterior) {
        __syncthreads();
        const int nc = 2 + d;
        for (int idx = tid; idx < Nfq * CW; idx += AS_THREADS) {
          int gf = idx / CW, col = c0 + idx % CW;
          int fp = f * Nfq + gf;
          const T* jb = tb.Jb + ((size_t)e * dm.m * dm.m + pair) * nc * Nfp + fp;
          T v = 0;
          if (col < Np) {
            v = jb[(size_t)Nfp] * tb.PhiF[(size_t)fp * Np + col];
            for (int l = 0; l < d; ++l) v -= jb[(size_t)(2 + l) * Nfp] * GlF[((size_t)l * Nfp + fp) * Np + col];
          } else if (col < ncol) {
            int t = col - Np;
            T mu = 0;
            const int* fl = tt.sfl + ((size_t)e * NbT + t) * 3;
            for (int q = 0; q < 3; ++q) {
              const int code = fl[q];
              if (code >= 0 && code / tt.NFS == f) mu = mutab[((size_t)f * Nfq + gf) * tt.NFS + code % tt.NFS];
            }
            v = jb[0] * mu;
            for (int l = 0; l < d; ++l) v += jb[(size_t)(2 + l) * Nfp] * HlF[((size_t)l * Nfp + fp) * NbT + t];
          }
          sV[idx] = v;
        }
        __syncthreads();
      }
      // trace rows: the slots living on this face, with the element's trace basis
      const int cnt = tt.nfs[e * dm.nf + f];
      const int* fsf = tt.fs + ((size_t)e * dm.nf + f) * tt.NFS;
      for (int idx = tid; idx < cnt * CW; idx += AS_THREADS) {
        int j = idx / CW, cc = idx % CW;
        T s = 0;
        for (int gf = 0; gf < Nfq; ++gf) s += mutab[((size_t)f * Nfq + gf) * tt.NFS + j] * sV[gf * CW + cc];
        tacc[fsf[j] * CW + cc] += s;
      }
    }
  }
  __syncthreads();

  // ---- write the element rows
  const int64_t nn = mix ? (int64_t)dm.nu + (int64_t)dm.m * Nb : dm.n;
  const int64_t ld = mix ? tt.ldv[e] : dm.ld;
  T* Se = mix ? S + tt.soff[e] : S + (LIST ? slot : e) * nn * ld;
  if (rhs64 != nullptr && pair == 0 && blockIdx.y == 0)
    for (int r = tid; r < nn; r += AS_THREADS) Se[r * ld + nn] = (T)rhs64[e * dm.n + r];
  auto colS = [&](int col) -> int64_t { return col < Np ? (int64_t)k * Np + col : (int64_t)dm.nu + (int64_t)k * Nb + (col - Np); };
  if (gemm_thread) {
    const T* Ms = tb.Mass + (size_t)e * Np * Np;
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      int row = trow * TM + a;
      if (row >= Np) continue;
      int sl = ref.slot[row];
#pragma unroll
      for (int b = 0; b < TN; ++b) {
        int col = c0 + tcol * TN + b;
        if (col >= ncol || col >= c0 + CW) continue;
        T v = acc[a][b];
        if (sl >= 0) v += facc[sl * CW + (col - c0)];
        if (i == k && col < Np) v += (T)ph.alpha * Ms[row * Np + col];
        Se[((int64_t)i * Np + row) * ld + colS(col)] = v;
      }
    }
  }
  for (int idx = tid; idx < Nb * CW; idx += AS_THREADS) {
    int s = idx / CW, col = c0 + idx % CW;
    if (col >= ncol) continue;
    Se[((int64_t)dm.nu + (int64_t)i * Nb + s) * ld + colS(col)] = tacc[idx];
  }
}

// ------------------------------------------------------------------ partial LU
// Right-looking blocked LU with partial pivoting of the bordered matrix, pivots
// only among the nu u-rows (largest |a|, smallest row on ties), eliminating the
// first nu columns from all n rows.  Afterwards rows [nu, n) x cols [nu, n] hold
// [K_e | R_e] = [Dt - Ct At^-1 Bt | Gt - Ct At^-1 Ft]; rows [0, nu) hold U (upper
// triangle, cols < nu) and L^-1 P [Bt Ft] (cols >= nu) for the back-substitution.
// T = float (mixed path) additionally writes back every panel in full (the
// multipliers L, in the row order of their own panel step) and the pivot rows, for
// the refinement solves.
// A[r][c] -= sum_j L[r][j] U[j][c] over rows [r_lo, r_hi), cols [c_lo, c_hi): L from the
// row-major panel P (row r at P[(r - kb) NB + j]), U = rows kb..kb+nb of A, staged by
// UCW-column chunks in Uc; 16 x 16 threads with 4 x 4 register tiles.
template <class T, int NB>
__device__ __forceinline__ void lu64_update_rect(T* __restrict__ A, int ld, const T* __restrict__ P,
                                                 T* __restrict__ Uc, int kb, int nb, int r_lo, int r_hi, int c_lo,
                                                 int c_hi) {
  const int tid = threadIdx.x;
  for (int cc = c_lo; cc < c_hi; cc += UCW) {
    const int cw = min(UCW, c_hi - cc);
    for (int idx = tid; idx < NB * UCW; idx += LU_THREADS) {
      int j = idx / UCW, c = idx % UCW;
      Uc[idx] = (j < nb && c < cw) ? A[(int64_t)(kb + j) * ld + cc + c] : (T)0;
    }
    __syncthreads();
    const int tc = tid % (UCW / 4), tr = tid / (UCW / 4);   // 16 x 16 threads, 4x4 tiles
    for (int rb = r_lo; rb < r_hi; rb += 64) {
      T a4[4][4];
      int rr[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        rr[a] = rb + tr * 4 + a;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          int c = tc * 4 + b;
          a4[a][b] = (rr[a] < r_hi && c < cw) ? A[(int64_t)rr[a] * ld + cc + c] : (T)0;
        }
      }
      for (int j = 0; j < nb; ++j) {
        T uv[4], lv[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) uv[b] = Uc[j * UCW + tc * 4 + b];
#pragma unroll
        for (int a = 0; a < 4; ++a) lv[a] = rr[a] < r_hi ? P[(rr[a] - kb) * NB + j] : (T)0;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) a4[a][b] = fma(-lv[a], uv[b], a4[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          int c = tc * 4 + b;
          if (rr[a] < r_hi && c < cw) A[(int64_t)rr[a] * ld + cc + c] = a4[a][b];
        }
    }
    __syncthreads();
  }
}

// |v| as a signed integer that orders like |v| (IEEE bit patterns of non-negative
// values are monotonic), -1 for NaN so that NaN is never chosen, like a floating-point
// comparison would; the pivot search of the FP64 LU then runs on the integer pipes
// instead of the slow FP64 pipe.
template <class T>
__device__ __forceinline__ long long abs_key(T v) {
  if constexpr (sizeof(T) == 8) {
    const long long k = __double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFLL;
    return k > 0x7FF0000000000000LL ? -1LL : k;
  } else {
    const long long k = (long long)(__float_as_int(v) & 0x7FFFFFFF);
    return k > 0x7F800000LL ? -1LL : k;
  }
}

// abs_key of +infinity: keys at or above it (and the -1 of NaN) are non-finite values
template <class T>
__device__ __forceinline__ long long inf_key() {
  if constexpr (sizeof(T) == 8) return 0x7FF0000000000000LL;
  else return 0x7F800000LL;
}

template <class T, int NB>
__device__ __forceinline__ void lu_element(const LuElem& el, T* __restrict__ S, int8_t* __restrict__ status,
                                           int* __restrict__ pivots, const int64_t e, bool defer_schur = false) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  __shared__ int piv[NB];
  __shared__ int perm[LU_MAX_NU];   // net row permutation of the current panel's interchanges
  __shared__ long long rv[LU_THREADS / 32];
  __shared__ int ri[LU_THREADS / 32];
  __shared__ int sing;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = el.n, nu = el.nu, ld = el.ld, ncol = n + 1;
  T* A = S + el.off;
  T* P = sm;                            // [n][NB]
  int nonfin = 0;                       // a pivot candidate was NaN or infinite
  T* Uc = P + (size_t)n * NB;           // [NB][UCW]
  if (tid == 0) sing = 0;
  for (int kb = 0; kb < nu; kb += NB) {
    const int nb = min(NB, nu - kb), rows = n - kb, prow = nu - kb;
    for (int idx = tid; idx < rows * NB; idx += LU_THREADS) {
      int r = idx / NB, j = idx % NB;
      P[idx] = j < nb ? A[(int64_t)(kb + r) * ld + kb + j] : (T)0;
    }
    for (int r = tid; r < prow; r += LU_THREADS) perm[r] = r;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
      long long best = -1;                  // largest |a| as an ordered integer key
      int bi = j;
      for (int r = j + tid; r < prow; r += LU_THREADS) {
        const long long v = abs_key(P[r * NB + j]);
        nonfin |= v < 0 || v >= inf_key<T>();
        if (v > best) { best = v; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
      __syncthreads();
      // every thread combines the warps' candidates (same order, same result)
      long long bk = rv[0];
      int pr = ri[0];
      for (int w = 1; w < LU_THREADS / 32; ++w) {
        const long long k = rv[w];
        if (k > bk || (k == bk && ri[w] < pr)) { bk = k; pr = ri[w]; }
      }
      if (bk <= 0) pr = j;                  // no nonzero candidate: singular
      if (tid == 0) {
        if (bk <= 0) sing = 1;
        piv[j] = pr;
        if (pivots) pivots[el.poff + kb + j] = kb + pr;
        if (pr != j) { const int t = perm[j]; perm[j] = perm[pr]; perm[pr] = t; }
      }
      if (pr != j && tid < NB) {
        T t = P[j * NB + tid];
        P[j * NB + tid] = P[pr * NB + tid];
        P[pr * NB + tid] = t;
      }
      __syncthreads();
      const T pv = P[j * NB + j];
      const T inv = pv != (T)0 ? (T)1 / pv : (T)0;
      for (int r = j + 1 + tid; r < rows; r += LU_THREADS) {
        T l = P[r * NB + j] * inv;
        P[r * NB + j] = l;
        for (int c = j + 1; c < nb; ++c) P[r * NB + c] = fma(-l, P[j * NB + c], P[r * NB + c]);
      }
      __syncthreads();
    }
    // U11 / L11 (and, when the factors are kept, L21) back to the element matrix
    const int wrows = (pivots || defer_schur) ? rows : nb;   // L21 is the W of the deferred form
    for (int idx = tid; idx < wrows * nb; idx += LU_THREADS) {
      int r = idx / nb, j = idx % nb;
      A[(int64_t)(kb + r) * ld + kb + j] = P[r * NB + j];
    }
    // trailing columns: row interchanges, then U12 = L11^-1 A12.  The panel's
    // interchanges leave row r holding the original row perm[r]; the rows below the
    // panel that change are pivot rows piv[j] >= nb and receive original rows above nb.
    // Each column gathers its new top rows (independent loads), moves the displaced
    // rows in groups of 8, then stores the top rows.
    for (int c = kb + nb + tid; c < ncol; c += LU_THREADS) {
      T x[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (j >= nb) break;
        x[j] = A[(int64_t)(kb + perm[j]) * ld + c];
      }
#pragma unroll
      for (int j0 = 0; j0 < NB; j0 += 8) {
        T y[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int r = j0 + j < nb ? piv[j0 + j] : 0;
          y[j] = (j0 + j < nb && r >= nb && perm[r] != r) ? A[(int64_t)(kb + perm[r]) * ld + c] : (T)0;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int r = j0 + j < nb ? piv[j0 + j] : 0;
          if (j0 + j < nb && r >= nb && perm[r] != r) A[(int64_t)(kb + r) * ld + c] = y[j];
        }
      }
      for (int j = 0; j < nb; ++j) {
        T s = x[j];
        for (int jj = 0; jj < j; ++jj) s = fma(-P[j * NB + jj], x[jj], s);
        x[j] = s;
        A[(int64_t)(kb + j) * ld + c] = s;
      }
    }
    __syncthreads();
    const int r0 = kb + nb;
    if (defer_schur) {
      // the trace block of the trace rows gets all panels at once afterwards
      lu64_update_rect<T, NB>(A, ld, P, Uc, kb, nb, r0, n, r0, nu);
      lu64_update_rect<T, NB>(A, ld, P, Uc, kb, nb, r0, nu, nu, ncol);
    } else {
      // A22 -= L21 U12, rows [kb+nb, n), cols [kb+nb, n]
      lu64_update_rect<T, NB>(A, ld, P, Uc, kb, nb, r0, n, r0, ncol);
    }
  }
  // status: a non-finite pivot candidate, an exact zero pivot, or a non-finite Schur
  // complement (deferred form: the caller checks the Schur complement after forming it)
  nonfin = __syncthreads_or(nonfin);
  if (defer_schur) {
    if (tid == 0) status[e] = nonfin ? IEDG_ELEM_NONFINITE : (sing ? IEDG_ELEM_SINGULAR : IEDG_ELEM_OK);
    __syncthreads();
    return;
  }
  int bad = 0;
  for (int idx = tid; idx < (n - nu) * (ncol - nu); idx += LU_THREADS) {
    int r = nu + idx / (ncol - nu), c = nu + idx % (ncol - nu);
    if (!isfinite(A[(int64_t)r * ld + c])) bad = 1;
  }
  bad = __syncthreads_or(bad);
  if (tid == 0)
    status[e] = nonfin ? IEDG_ELEM_NONFINITE
                       : (sing ? IEDG_ELEM_SINGULAR : (bad ? IEDG_ELEM_NONFINITE : IEDG_ELEM_OK));
}

// ----------------------------------------------------------- FP64 Schur complement on tcgen05
// [K | R] = [D | G] - W [Z | z] of the FP64 form with the products on the tensor cores,
// by an exact splitting of the FP64 operands (the Ozaki scheme): each row i of W is
// scaled by a power of two 2^e_i >= its largest entry, each column j of Z by 2^f_j,
// and the scaled entries are written as sums of OZ_S integer slices of OZ_BETA bits,
//   W_ik = 2^e_i sum_s v_s 2^(-s beta),  Z_kj = 2^f_j sum_t w_t 2^(-t beta)  (+ a rest
// below 2^-(S beta)), v, w integers with |v|, |w| <= 2^beta, exact in TF32.  The slice
// products of one level l = s + t (2 <= l <= S + 1) share the scale 2^(e_i + f_j - l beta)
// and accumulate in one FP32 TMEM accumulator: with beta = 7 and K chunks of 64 every
// partial sum is an integer below 2^23, so the tensor cores add exactly; each chunk's
// levels are then scaled and summed in FP64.  Levels above S + 1 (below 2^-63 of the
// product scale) are dropped.  The splitting and the level sums are FP64 work
// (about a quarter of the FP64 multiply-adds the product itself would take).
constexpr int OZ_S = 8, OZ_BETA = 7, OZ_L = 8;           // slices, bits per slice, levels 2..9
constexpr int OZ_KC = 64, OZ_KS = 16;                    // exact-accumulation chunk, staging step
constexpr int OZ_TM = 128, OZ_TN = 32;
constexpr int OZ_TMEM_COLS = OZ_L * OZ_TN;              // 256
constexpr int OZ_A_BYTES = OZ_TM * OZ_KS * 4, OZ_B_BYTES = OZ_TN * OZ_KS * 4;
constexpr int OZ_STAGE_BYTES = OZ_S * (OZ_A_BYTES + OZ_B_BYTES);   // 80 KB

// Scratch of one CTA for the slices and scales of its current element.
struct OzScratch {
  float* ws;      // [S][nt][nu]      slices of W, K contiguous
  float* zs;      // [S][nt + 1][nu]  slices of Z^T, K contiguous
  double* rs;     // [nt]             2^e_i
  double* cs;     // [nt + 1]         2^f_j
};

__device__ __forceinline__ double pow2_at_least(double m) {
  if (!(m > 0.0)) return 1.0;
  int ex;
  frexp(m, &ex);                  // m = f 2^ex, f in [0.5, 1): m < 2^ex
  return ldexp(1.0, ex);
}

__device__ void oz_split(const double* __restrict__ A, int ld, int n, int nu, const OzScratch& sc) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = LU_THREADS / 32;
  const int nt = n - nu, nt1 = nt + 1;
  // row scales of W (one warp per row) and column scales of Z (one thread per column)
  for (int i = warp; i < nt; i += nw) {
    const double* row = A + (int64_t)(nu + i) * ld;
    double mx = 0.0;
    for (int k = lane; k < nu; k += 32) mx = fmax(mx, fabs(row[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) sc.rs[i] = pow2_at_least(mx);
  }
  for (int j = tid; j < nt1; j += LU_THREADS) {
    double mx = 0.0;
    for (int k = 0; k < nu; ++k) mx = fmax(mx, fabs(A[(int64_t)k * ld + nu + j]));
    sc.cs[j] = pow2_at_least(mx);
  }
  __syncthreads();
  const double up = ldexp(1.0, OZ_BETA);
  for (int idx = tid; idx < nt * nu; idx += LU_THREADS) {
    const int i = idx / nu, k = idx % nu;
    double x = A[(int64_t)(nu + i) * ld + k] / sc.rs[i];          // exact: power of two
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      const double t = x * up;
      const double v = rint(t);
      x = t - v;
      sc.ws[((size_t)s * nt + i) * nu + k] = (float)v;
    }
  }
  for (int idx = tid; idx < nt1 * nu; idx += LU_THREADS) {
    const int k = idx / nt1, j = idx % nt1;
    double x = A[(int64_t)k * ld + nu + j] / sc.cs[j];
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      const double t = x * up;
      const double v = rint(t);
      x = t - v;
      sc.zs[((size_t)s * nt1 + j) * nu + k] = (float)v;
    }
  }
  __syncthreads();
}

// Stage K columns k0 .. k0+15 of every slice of the tile's W rows and Z columns.
__device__ __forceinline__ void oz_stage(const OzScratch& sc, int nt, int nu, int rt, int ct, int k0, char* stage) {
  const int tid = threadIdx.x, nt1 = nt + 1;
  char* sa = stage;
  char* sb = stage + OZ_S * OZ_A_BYTES;
  for (int idx = tid; idx < OZ_S * OZ_TM * OZ_KS; idx += LU_THREADS) {
    const int s = idx / (OZ_TM * OZ_KS), r = (idx / OZ_KS) % OZ_TM, k = idx % OZ_KS;
    const int i = rt + r, kk = k0 + k;
    const float v = (i < nt && kk < nu) ? sc.ws[((size_t)s * nt + i) * nu + kk] : 0.f;
    const uint32_t off = (uint32_t)((r >> 3) * (OZ_KS / 4) * 128 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
    *reinterpret_cast<float*>(sa + s * OZ_A_BYTES + off) = v;
  }
  for (int idx = tid; idx < OZ_S * OZ_TN * OZ_KS; idx += LU_THREADS) {
    const int s = idx / (OZ_TN * OZ_KS), r = (idx / OZ_KS) % OZ_TN, k = idx % OZ_KS;
    const int j = ct + r, kk = k0 + k;
    const float v = (j < nt1 && kk < nu) ? sc.zs[((size_t)s * nt1 + j) * nu + kk] : 0.f;
    const uint32_t off = (uint32_t)((r >> 3) * (OZ_KS / 4) * 128 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
    *reinterpret_cast<float*>(sb + s * OZ_B_BYTES + off) = v;
  }
}

// One thread: every slice pair of levels 2..S+1 for the staged K step; level l goes
// to TMEM columns (l - 2) OZ_TN ..; `first` starts the chunk's accumulators.
__device__ __forceinline__ void oz_issue(uint32_t tmem, const char* stage, bool first) {
  const uint32_t a0 = tc::smem_u32(stage), b0 = a0 + OZ_S * OZ_A_BYTES;
  constexpr uint32_t IDESC = tc::idesc_tf32(OZ_TM, OZ_TN);
  constexpr uint32_t SBO = (OZ_KS / 4) * 128;
  for (int s = 1; s <= OZ_S; ++s)
    for (int t = 1; t <= OZ_S; ++t) {
      const int l = s + t;
      if (l > OZ_L + 1) continue;
      const uint32_t d = tmem + (uint32_t)((l - 2) * OZ_TN);
      // the first product of a level in the chunk is the one with s = 1
#pragma unroll
      for (int kst = 0; kst < OZ_KS / 8; ++kst) {
        const uint32_t ko = kst * 256;
        const bool acc = !(first && s == 1 && kst == 0);
        tc::mma_tf32(d, tc::desc_kmajor(a0 + (s - 1) * OZ_A_BYTES + ko, 128, SBO),
                     tc::desc_kmajor(b0 + (t - 1) * OZ_B_BYTES + ko, 128, SBO), IDESC, acc ? 1u : 0u);
      }
    }
}

__device__ void schur_ozaki(double* __restrict__ A, int ld, int n, int nu, const OzScratch& sc, char* smem,
                            TcState* tcs) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nt = n - nu, ncol = n + 1;
  const int q = warp & 3, h = warp >> 2;
  oz_split(A, ld, n, nu, sc);
  for (int rt = 0; rt < nt && !tcs->failed; rt += OZ_TM) {
    for (int ct = 0; ct < ncol - nu && !tcs->failed; ct += OZ_TN) {
      for (int kc = 0; kc < nu && !tcs->failed; kc += OZ_KC) {
        for (int k0 = kc; k0 < min(kc + OZ_KC, nu); k0 += OZ_KS) {
          oz_stage(sc, nt, nu, rt, ct, k0, smem);
          tc::fence_proxy_async();
          __syncthreads();
          tc::fence_after_sync();
          if (tid == 0) {
            oz_issue(tcs->tmem, smem, k0 == kc);
            tc::mma_commit(tcs->mbar);
          }
          tcs->pending[0] = 1;
          const bool ok = __syncthreads_and(tc::mbar_wait(tcs->mbar, tcs->phase[0], tcs->limit));
          if (!ok) { tcs->failed = 1; break; }
          tcs->phase[0] ^= 1u;
          tcs->pending[0] = 0;
          tc::fence_after_sync();
        }
        if (tcs->failed) break;
        // epilogue: warp (q, h) owns rows 32 q .. 32 q + 31 and columns 16 h .. 16 h + 15
        const int i = rt + 32 * q + lane;
        const double rsc = i < nt ? sc.rs[i] : 0.0;
#pragma unroll 1
        for (int c8 = 0; c8 < 2; ++c8) {
          const int c0 = 16 * h + 8 * c8;
          double sum[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) sum[j] = 0.0;
#pragma unroll 1
          for (int l = 0; l < OZ_L; ++l) {
            float v8[8];
            tc::tmem_ld8(tcs->tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(l * OZ_TN + c0), v8);
            const double w = ldexp(1.0, -(l + 2) * OZ_BETA);
#pragma unroll
            for (int j = 0; j < 8; ++j) sum[j] = fma((double)v8[j], w, sum[j]);
          }
          if (i >= nt) continue;
          double* dst = A + (int64_t)(nu + i) * ld + nu + ct + c0;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int jj = ct + c0 + j;
            if (jj < ncol - nu) dst[j] -= (rsc * sc.cs[jj]) * sum[j];
          }
        }
        tc::fence_before_sync();
        __syncthreads();
      }
    }
  }
}

// FP32 partial LU for the mixed path.  Same algorithm and pivot rule as k_lu, with
// the panel kept column-major in shared memory (contiguous rows for the pivot search,
// the elimination and vector loads of L21) and a 4 x 8 register tile per thread in
// the trailing update (float4 loads: three shared loads per 32 multiply-adds), so the
// update runs at FFMA rather than shared-memory rate, with two CTAs per SM.  The full panel (L) and the
// pivot rows are written back for the refinement solves.
constexpr int L32_NB = 32;
constexpr int L32_UCW = 128;      // trailing-update column chunk
constexpr int L32_TM = 4, L32_TN = 8;


// The 4 x 8 tile of A at rows rr0.., columns cc + tc * 8.. (zero outside the update).
__device__ __forceinline__ void lu32_load_tile(const float* __restrict__ A, int ld, int rr0, int r_hi, int cc, int tc,
                                               int cw, bool cvec, float (&t)[L32_TM][L32_TN]) {
#pragma unroll
  for (int a = 0; a < L32_TM; ++a) {
    const int rr = rr0 + a;
    if (cvec && rr < r_hi) {
      const float4* src = reinterpret_cast<const float4*>(A + (int64_t)rr * ld + cc + tc * L32_TN);
      const float4 v0 = src[0], v1 = src[1];
      t[a][0] = v0.x; t[a][1] = v0.y; t[a][2] = v0.z; t[a][3] = v0.w;
      t[a][4] = v1.x; t[a][5] = v1.y; t[a][6] = v1.z; t[a][7] = v1.w;
    } else {
#pragma unroll
      for (int b = 0; b < L32_TN; ++b) {
        const int c = tc * L32_TN + b;
        t[a][b] = (rr < r_hi && c < cw) ? A[(int64_t)rr * ld + cc + c] : 0.f;
      }
    }
  }
}

// Ask L2 for the lines of the 4 x 8 tile at rows rr0.. (no registers held).
__device__ __forceinline__ void lu32_prefetch_tile(const float* __restrict__ A, int ld, int rr0, int r_hi, int cc,
                                                   int tc) {
#pragma unroll
  for (int a = 0; a < L32_TM; ++a)
    if (rr0 + a < r_hi)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(A + (int64_t)(rr0 + a) * ld + cc + tc * L32_TN));
}

// A[r][c] -= sum_j L[r][j] U[j][c] over rows [r_lo, r_hi), cols [c_lo, c_hi): L from the
// column-major panel P (row r at P[j n + r - kb]), U = rows kb..kb+nb of A.  4 x 8
// register tiles, U staged in Uc by 128-column chunks; the next row block's tile is
// requested from L2 while the current one is updated.  Columns past c_hi are written
// back unchanged only when they are padding of the row (c_hi = n + 1).
__device__ __forceinline__ void lu32_update_rect(float* __restrict__ A, int ld, int n, const float* __restrict__ P,
                                                 float* __restrict__ Uc, int kb, int nb, int r_lo, int r_hi,
                                                 int c_lo, int c_hi) {
  const int tid = threadIdx.x;
  const bool vec = ((nb & 3) == 0) && ((n & 3) == 0);
  const int tc = tid % (L32_UCW / L32_TN), tr = tid / (L32_UCW / L32_TN);   // 16 x 16
  const int vlim = (c_hi == n + 1) ? ld : c_hi;     // last column a vector access may touch
  constexpr int RB = 16 * L32_TM;                   // rows per block of the CTA
  for (int cc = c_lo; cc < c_hi; cc += L32_UCW) {
    const int cw = min(L32_UCW, c_hi - cc);
    for (int idx = tid; idx < L32_NB * L32_UCW; idx += LU_THREADS) {
      int j = idx / L32_UCW, c = idx % L32_UCW;
      Uc[idx] = (j < nb && c < cw) ? A[(int64_t)(kb + j) * ld + cc + c] : 0.f;
    }
    __syncthreads();
    const bool cvec = ((cc & 3) == 0) && (cc + tc * L32_TN + L32_TN <= vlim);
    for (int rb = r_lo; rb < r_hi; rb += RB) {
      const int rr0 = rb + tr * L32_TM;
      float acc[L32_TM][L32_TN];
      lu32_load_tile(A, ld, rr0, r_hi, cc, tc, cw, cvec, acc);
      if (rb + RB < r_hi) lu32_prefetch_tile(A, ld, rr0 + RB, r_hi, cc, tc);
      if (nb == L32_NB && vec && rr0 + L32_TM <= r_hi) {
        // full panel, whole tile: fixed trip count and no per-step bounds tests
        const float* lp = P + (rr0 - kb);
        const float* up = Uc + tc * L32_TN;
#pragma unroll 2
        for (int j = 0; j < L32_NB; ++j) {
          const float4 l0 = *reinterpret_cast<const float4*>(lp + j * n);
          const float4 u0 = *reinterpret_cast<const float4*>(up + j * L32_UCW);
          const float4 u1 = *reinterpret_cast<const float4*>(up + j * L32_UCW + 4);
          const float lv[L32_TM] = {l0.x, l0.y, l0.z, l0.w};
          const float uv[L32_TN] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
          for (int a = 0; a < L32_TM; ++a)
#pragma unroll
            for (int b = 0; b < L32_TN; ++b) acc[a][b] = fmaf(-lv[a], uv[b], acc[a][b]);
        }
      } else if (rr0 < r_hi) {
#pragma unroll 4
        for (int j = 0; j < nb; ++j) {
          float lv[L32_TM], uv[L32_TN];
          const float* lp = P + j * n + (rr0 - kb);
          if (vec && rr0 + L32_TM <= r_hi) {
            float4 l0 = *reinterpret_cast<const float4*>(lp);
            lv[0] = l0.x; lv[1] = l0.y; lv[2] = l0.z; lv[3] = l0.w;
          } else {
#pragma unroll
            for (int a = 0; a < L32_TM; ++a) lv[a] = (rr0 + a < r_hi) ? lp[a] : 0.f;
          }
          const float4 u0 = *reinterpret_cast<const float4*>(Uc + j * L32_UCW + tc * L32_TN);
          const float4 u1 = *reinterpret_cast<const float4*>(Uc + j * L32_UCW + tc * L32_TN + 4);
          uv[0] = u0.x; uv[1] = u0.y; uv[2] = u0.z; uv[3] = u0.w;
          uv[4] = u1.x; uv[5] = u1.y; uv[6] = u1.z; uv[7] = u1.w;
#pragma unroll
          for (int a = 0; a < L32_TM; ++a)
#pragma unroll
            for (int b = 0; b < L32_TN; ++b) acc[a][b] = fmaf(-lv[a], uv[b], acc[a][b]);
        }
      }
#pragma unroll
      for (int a = 0; a < L32_TM; ++a) {
        const int rr = rr0 + a;
        if (cvec && rr < r_hi) {
          float4* dst = reinterpret_cast<float4*>(A + (int64_t)rr * ld + cc + tc * L32_TN);
          dst[0] = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
          dst[1] = make_float4(acc[a][4], acc[a][5], acc[a][6], acc[a][7]);
        } else {
#pragma unroll
          for (int b = 0; b < L32_TN; ++b) {
            int c = tc * L32_TN + b;
            if (rr < r_hi && c < cw) A[(int64_t)rr * ld + cc + c] = acc[a][b];
          }
        }
      }
    }
    __syncthreads();
  }
}

// Deferred Schur complement on the tensor cores: [K | R] = [D | G] - W [Z | z] for rows
// [nu, n) and columns [nu, n], W = A[nu:n, 0:nu] (the eliminated trace rows, L21 of
// every panel) and Z = A[0:nu, nu:n] (U12 of every panel), so K accumulates over the
// whole K = nu in TMEM and the trace block is read and written once.  128 x 64 output
// tiles, K chunks of 32 in two operand stages so that one chunk is staged while the
// tensor core works on the other; one thread issues the MMAs, completion through
// per-stage mbarriers with bounded waits; the epilogue reads TMEM with all eight warps.
// Operand forms (KIND): kSchurFp32 = TF32 high and low parts, three products (hi hi +
// hi lo + lo hi, FP32 accuracy, 48 KB stages); kSchurTf32 = one product of the operands
// rounded to TF32 (24 KB); kSchurBf16 = one product of BF16 operands (12 KB).  All
// accumulate in FP32.
constexpr int TC_TM = 128, TC_TN = 64, TC_KC = 32;
constexpr int TC_STAGE_BYTES = 2 * TC_TM * TC_KC * 4 + 2 * TC_TN * TC_KC * 4;   // 48 KB, the largest form

template <int KIND>
struct SchurForm {
  static constexpr int EB = KIND == kSchurBf16 ? 2 : 4;          // bytes per operand value
  static constexpr int PARTS = KIND == kSchurFp32 ? 2 : 1;       // hi (+ lo)
  static constexpr int A_BYTES = TC_TM * TC_KC * EB, B_BYTES = TC_TN * TC_KC * EB;
  static constexpr int SBO = TC_KC * EB / 16 * 128;               // 8-row group stride
  __device__ static uint32_t off(int row, int k) { return EB == 4 ? tc::core_off32(row, k) : tc::core_off16(row, k); }
  // value v at (row, k) of the A (b = false) or B operand tile
  __device__ static void put(char* stage, bool b, int row, int k, float v) {
    char* base = stage + (b ? PARTS * A_BYTES : 0);
    const uint32_t o = off(row, k);
    if constexpr (KIND == kSchurFp32) {
      float hi, lo;
      tc::split_tf32(v, hi, lo);
      *reinterpret_cast<float*>(base + o) = hi;
      *reinterpret_cast<float*>(base + (b ? B_BYTES : A_BYTES) + o) = lo;
    } else if constexpr (KIND == kSchurTf32) {
      *reinterpret_cast<float*>(base + o) = tc::round_tf32(v);
    } else {
      *reinterpret_cast<__nv_bfloat16*>(base + o) = __float2bfloat16_rn(v);
    }
  }
};

template <int KIND>
__device__ __forceinline__ void schur_stage(const float* __restrict__ A, int ld, int n, int nu, int ncol, int rt,
                                            int ct, int kc, char* stage) {
  using F = SchurForm<KIND>;
  const int tid = threadIdx.x;
  // A operand: W rows rt .. rt+127, K columns kc .. kc+31 (k fastest: coalesced rows)
  for (int idx = tid; idx < TC_TM * TC_KC; idx += LU_THREADS) {
    const int mm = idx >> 5, k = idx & 31;
    const int r = rt + mm, c = kc + k;
    F::put(stage, false, mm, k, (r < n && c < nu) ? A[(int64_t)r * ld + c] : 0.f);
  }
  // B operand (N x K, K-major): Z rows kc .. kc+31, columns ct .. ct+63 (column fastest)
  for (int idx = tid; idx < TC_TN * TC_KC; idx += LU_THREADS) {
    const int k = idx >> 6, nn = idx & 63;
    const int r = kc + k, c = ct + nn;
    F::put(stage, true, nn, k, (r < nu && c < ncol) ? A[(int64_t)r * ld + c] : 0.f);
  }
}

template <int KIND>
__device__ __forceinline__ void schur_issue(uint32_t tmem, const char* stage, bool first) {
  using F = SchurForm<KIND>;
  const uint32_t aH = tc::smem_u32(stage), aL = aH + F::A_BYTES;
  const uint32_t bH = aH + F::PARTS * F::A_BYTES, bL = bH + F::B_BYTES;
  // one instruction covers 32 bytes of K (8 TF32 or 16 BF16 values): two core matrices
#pragma unroll
  for (int st = 0; st < TC_KC * F::EB / 32; ++st) {
    const uint32_t ko = st * 256, acc = (first && st == 0) ? 0u : 1u;
    if constexpr (KIND == kSchurBf16) {
      constexpr uint32_t IDESC = tc::idesc_bf16(TC_TM, TC_TN);
      tc::mma_bf16(tmem, tc::desc_kmajor(aH + ko, 128, F::SBO), tc::desc_kmajor(bH + ko, 128, F::SBO), IDESC, acc);
    } else {
      constexpr uint32_t IDESC = tc::idesc_tf32(TC_TM, TC_TN);
      tc::mma_tf32(tmem, tc::desc_kmajor(aH + ko, 128, F::SBO), tc::desc_kmajor(bH + ko, 128, F::SBO), IDESC, acc);
      if constexpr (KIND == kSchurFp32) {
        tc::mma_tf32(tmem, tc::desc_kmajor(aH + ko, 128, F::SBO), tc::desc_kmajor(bL + ko, 128, F::SBO), IDESC, 1);
        tc::mma_tf32(tmem, tc::desc_kmajor(aL + ko, 128, F::SBO), tc::desc_kmajor(bH + ko, 128, F::SBO), IDESC, 1);
      }
    }
  }
}

// Bounded wait on stage b's barrier by every thread; the outcome is made uniform.
// (A wait that ran out leaves the phase where it was, so the drain can wait for it.)
__device__ __forceinline__ bool schur_wait(TcState* tcs, int b) {
  const bool ok = __syncthreads_and(tc::mbar_wait(tcs->mbar + b, tcs->phase[b], tcs->limit));
  if (ok) { tcs->phase[b] ^= 1u; tcs->pending[b] = 0; }
  else tcs->failed = 1;
  return ok;
}

template <int KIND>
__device__ void schur_tc(float* __restrict__ A, int ld, int n, int nu, char* smem, TcState* tcs) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ncol = n + 1;
  const int nk = (nu + TC_KC - 1) / TC_KC;
  const int q = warp & 3, h = warp >> 2;
  for (int rt = nu; rt < n && !tcs->failed; rt += TC_TM) {
    for (int ct = nu; ct < ncol && !tcs->failed; ct += TC_TN) {
      schur_stage<KIND>(A, ld, n, nu, ncol, rt, ct, 0, smem);
      tc::fence_proxy_async();
      __syncthreads();
      tc::fence_after_sync();
      for (int c = 0; c < nk; ++c) {
        const int b = c & 1;
        if (tid == 0) {
          schur_issue<KIND>(tcs->tmem, smem + b * TC_STAGE_BYTES, c == 0);
          tc::mma_commit(tcs->mbar + b);
        }
        tcs->pending[b] = 1;
        if (c + 1 < nk) {
          // the other stage was last read by the MMAs of chunk c - 1
          if (c >= 1 && !schur_wait(tcs, b ^ 1)) break;
          schur_stage<KIND>(A, ld, n, nu, ncol, rt, ct, (c + 1) * TC_KC, smem + (b ^ 1) * TC_STAGE_BYTES);
          tc::fence_proxy_async();
          __syncthreads();
          tc::fence_after_sync();
        }
      }
      if (tcs->failed) break;
      // the two commits not waited for yet: chunks nk - 2 and nk - 1
      if (nk >= 2 && !schur_wait(tcs, (nk - 2) & 1)) break;
      if (!schur_wait(tcs, (nk - 1) & 1)) break;
      tc::fence_after_sync();
      // epilogue: warp (q, h) owns rows 32 q .. 32 q + 31 and columns 32 h .. 32 h + 31
      const int row = rt + 32 * q + lane;
#pragma unroll 1
      for (int c8 = 0; c8 < 4; ++c8) {
        const int c0 = 32 * h + 8 * c8;
        float pv8[8];
        tc::tmem_ld8(tcs->tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, pv8);
        if (row >= n || ct + c0 >= ncol) continue;
        float* dst = A + (int64_t)row * ld + ct + c0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (ct + c0 + j < ncol) dst[j] -= pv8[j];
      }
      tc::fence_before_sync();
      __syncthreads();
    }
  }
}

template <bool TC, int KIND = kSchurFp32>
__device__ __forceinline__ void lu32_element(const LuElem& el, float* __restrict__ S, int8_t* __restrict__ status,
                                             int* __restrict__ pivots, const int64_t e, TcState* tcs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* P = reinterpret_cast<float*>(smraw);          // [NB][n] column-major panel
  float* Uc = P + (size_t)L32_NB * el.n;                // [NB][UCW]
  __shared__ int piv[L32_NB];
  __shared__ int perm[LU_MAX_NU];   // net row permutation of the current panel's interchanges
  __shared__ float rv[LU_THREADS / 32];
  __shared__ int ri[LU_THREADS / 32];
  __shared__ int sing;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = el.n, nu = el.nu, ld = el.ld, ncol = n + 1;
  float* A = S + el.off;
  int nonfin = 0;                       // a pivot candidate was NaN or infinite
  if (tid == 0) sing = 0;
  for (int kb = 0; kb < nu; kb += L32_NB) {
    const int nb = min(L32_NB, nu - kb), rows = n - kb, prow = nu - kb;
    for (int idx = tid; idx < rows * L32_NB; idx += LU_THREADS) {
      int r = idx / L32_NB, j = idx % L32_NB;
      P[j * n + r] = j < nb ? A[(int64_t)(kb + r) * ld + kb + j] : 0.f;
    }
    for (int r = tid; r < prow; r += LU_THREADS) perm[r] = r;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
      const float* Pj = P + j * n;
      float best = -1.f;
      int bi = j;
      for (int r = j + tid; r < prow; r += LU_THREADS) {
        float v = fabsf(Pj[r]);
        nonfin |= !(v <= 3.402823466e38f);
        if (v > best) { best = v; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
      __syncthreads();
      // every thread combines the warps' candidates (same order, same result)
      float bv = rv[0];
      int pr = ri[0];
      for (int w = 1; w < LU_THREADS / 32; ++w)
        if (rv[w] > bv || (rv[w] == bv && ri[w] < pr)) { bv = rv[w]; pr = ri[w]; }
      if (!(bv > 0.f)) pr = j;
      if (tid == 0) {
        if (!(bv > 0.f)) sing = 1;
        piv[j] = pr;
        pivots[el.poff + kb + j] = kb + pr;
        if (pr != j) { const int t = perm[j]; perm[j] = perm[pr]; perm[pr] = t; }
      }
      if (pr != j && tid < L32_NB) {
        float t = P[tid * n + j];
        P[tid * n + j] = P[tid * n + pr];
        P[tid * n + pr] = t;
      }
      __syncthreads();
      const float pv = Pj[j];
      const float inv = pv != 0.f ? 1.f / pv : 0.f;
      for (int r = j + 1 + tid; r < rows; r += LU_THREADS) {
        float l = Pj[r] * inv;
        P[j * n + r] = l;
        for (int c = j + 1; c < nb; ++c) P[c * n + r] = fmaf(-l, P[c * n + j], P[c * n + r]);
      }
      __syncthreads();
    }
    // full panel back (U11, L11, L21): needed by the refinement solves
    for (int idx = tid; idx < rows * nb; idx += LU_THREADS) {
      int r = idx / nb, j = idx % nb;
      A[(int64_t)(kb + r) * ld + kb + j] = P[j * n + r];
    }
    // trailing columns: row interchanges, then U12 = L11^-1 A12.  The panel's
    // interchanges, applied in order, leave row r holding the original row perm[r]; the
    // rows below the panel that change are among the pivot rows piv[j] >= nb, and they
    // receive original rows above nb.  Each column gathers its new top rows first
    // (independent loads), then moves the displaced rows, then stores the top rows.
    for (int c = kb + nb + tid; c < ncol; c += LU_THREADS) {
      float x[L32_NB];
#pragma unroll
      for (int j = 0; j < L32_NB; ++j) {
        if (j >= nb) break;
        x[j] = A[(int64_t)(kb + perm[j]) * ld + c];
      }
      // displaced rows take original top rows (unchanged until the stores below), in
      // groups of 8 loads before their stores
#pragma unroll
      for (int j0 = 0; j0 < L32_NB; j0 += 8) {
        float y[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int r = j0 + j < nb ? piv[j0 + j] : 0;
          y[j] = (j0 + j < nb && r >= nb && perm[r] != r) ? A[(int64_t)(kb + perm[r]) * ld + c] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int r = j0 + j < nb ? piv[j0 + j] : 0;
          if (j0 + j < nb && r >= nb && perm[r] != r) A[(int64_t)(kb + r) * ld + c] = y[j];
        }
      }
#pragma unroll
      for (int j = 0; j < L32_NB; ++j) {
        if (j >= nb) break;
        float s = x[j];
#pragma unroll
        for (int jj = 0; jj < L32_NB; ++jj) {
          if (jj >= j) break;
          s = fmaf(-P[jj * n + j], x[jj], s);
        }
        x[j] = s;
        A[(int64_t)(kb + j) * ld + c] = s;
      }
    }
    __syncthreads();
    const int r0 = kb + nb;
    if constexpr (TC) {
      // deferred Schur complement: the u-columns of every row and the trace columns of
      // the u-rows are updated now (the next panels and U12 need them); the trace block
      // of the trace rows receives all panels at once on the tensor cores below
      lu32_update_rect(A, ld, n, P, Uc, kb, nb, r0, n, r0, nu);
      lu32_update_rect(A, ld, n, P, Uc, kb, nb, r0, nu, nu, ncol);
    } else {
      // A22 -= L21 U12, rows [kb+nb, n), cols [kb+nb, n]
      lu32_update_rect(A, ld, n, P, Uc, kb, nb, r0, n, r0, ncol);
    }
  }
  if constexpr (TC) {
    __syncthreads();
    schur_tc<KIND>(A, ld, n, nu, reinterpret_cast<char*>(smraw), tcs);     // the panel buffer is free now
  }
  __syncthreads();
  int bad = 0;
  for (int idx = tid; idx < (n - nu) * (ncol - nu); idx += LU_THREADS) {
    int r = nu + idx / (ncol - nu), c = nu + idx % (ncol - nu);
    if (!isfinite(A[(int64_t)r * ld + c])) bad = 1;
  }
  bad = __syncthreads_or(bad);
  nonfin = __syncthreads_or(nonfin);
  if (tid == 0) {
    if (TC && tcs->failed) status[e] = IEDG_ELEM_TIMEOUT;
    else status[e] = nonfin ? IEDG_ELEM_NONFINITE
                            : (sing ? IEDG_ELEM_SINGULAR : (bad ? IEDG_ELEM_NONFINITE : IEDG_ELEM_OK));
  }
}

template <class T, int NB>
__global__ void __launch_bounds__(LU_THREADS)
k_lu(Dims dm, LuDesc lud, T* __restrict__ S, int8_t* __restrict__ status, int* __restrict__ pivots, int64_t* queue,
     int64_t E, const int64_t* __restrict__ active = nullptr) {
  int64_t e;
  for (int64_t it = 0; next_element(queue, E, it, lud.order, &e); ++it)
    if (active == nullptr || active[e] >= 0) lu_element<T, NB>(lu_elem(dm, lud, e), S, status, pivots, e);
}

__global__ void __launch_bounds__(LU_THREADS, 2)
k_lu32(Dims dm, LuDesc lud, float* __restrict__ S, int8_t* __restrict__ status, int* __restrict__ pivots,
       int64_t* queue, int64_t E) {
  int64_t e;
  for (int64_t it = 0; next_element(queue, E, it, lud.order, &e); ++it)
    lu32_element<false>(lu_elem(dm, lud, e), S, status, pivots, e, nullptr);
}

// Tensor-core form: TMEM (128 columns) and the completion barrier are set up once per
// CTA; a CTA whose completion wait ran out stops taking elements, waits once more
// (bounded) for its MMAs, and frees its TMEM.
template <int KIND>
__global__ void __launch_bounds__(LU_THREADS, 2)
k_lu32_tc(Dims dm, LuDesc lud, float* __restrict__ S, int8_t* __restrict__ status, int* __restrict__ pivots,
          int64_t* queue, int64_t E, int* err, int wait_limit) {
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ TcState tcs;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, TC_TN);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0) {
    tcs.tmem = tmem_base;
    tcs.mbar = mbar;
    tcs.phase[0] = 0;
    tcs.phase[1] = 0;
    tcs.failed = 0;
    tcs.limit = wait_limit;
    tcs.pending[0] = 0;
    tcs.pending[1] = 0;
  }
  __syncthreads();
  // each thread keeps its own copy of the phases; the shared copy is only the start
  TcState mine = tcs;
  int64_t e;
  int64_t it = 0;
  for (; next_element(queue, E, it, lud.order, &e); ++it) {
    lu32_element<true, KIND>(lu_elem(dm, lud, e), S, status, pivots, e, &mine);
    if (__syncthreads_or(mine.failed)) {
      if (tid == 0) atomicOr(err, 1);
      tc_drain(mine);     // MMAs still in flight finish before the TMEM is freed
      ++it;
      break;
    }
  }
  // after a failed wait this CTA factors nothing more: the elements it still takes from
  // the queue are flagged, so no element is left unfactored with an OK status
  if (mine.failed)
    for (; next_element(queue, E, it, lud.order, &e); ++it)
      if (tid == 0) status[e] = IEDG_ELEM_TIMEOUT;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem_base, TC_TN);
}

// FP64 partial LU with the Schur complement on the tensor cores (schur_ozaki).  The CTA
// holds 256 TMEM columns (two resident CTAs fit an SM's 512) and one completion barrier.
__global__ void __launch_bounds__(LU_THREADS)
k_lu64_oz(Dims dm, LuDesc lud, double* __restrict__ S, int8_t* __restrict__ status, int64_t* queue, int64_t E,
          float* __restrict__ scratch, int64_t scratch_floats, int* err, int wait_limit) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ TcState tcs;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, OZ_TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&mbar[0], 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0) {
    tcs.tmem = tmem_base;
    tcs.mbar = mbar;
    tcs.phase[0] = 0;
    tcs.phase[1] = 0;
    tcs.failed = 0;
    tcs.limit = wait_limit;
    tcs.pending[0] = 0;
    tcs.pending[1] = 0;
  }
  __syncthreads();
  TcState mine = tcs;
  // this CTA's slices and scales
  float* base = scratch + (size_t)blockIdx.x * scratch_floats;
  OzScratch sc;
  {
    const size_t ntm = dm.nt + 1, num = dm.nu;
    sc.ws = base;
    sc.zs = sc.ws + (size_t)OZ_S * ntm * num;
    double* dd = reinterpret_cast<double*>(sc.zs + (size_t)OZ_S * ntm * num);
    sc.rs = dd;
    sc.cs = dd + ntm;
  }
  int64_t e;
  int64_t it = 0;
  for (; next_element(queue, E, it, lud.order, &e); ++it) {
    const LuElem el = lu_elem(dm, lud, e);
    lu_element<double, 16>(el, S, status, nullptr, e, true);
    schur_ozaki(S + el.off, el.ld, el.n, el.nu, sc, reinterpret_cast<char*>(smraw), &mine);
    // non-finite Schur complement
    double* A = S + el.off;
    const int n = el.n, nu = el.nu, ncol = n + 1;
    int bad = 0;
    for (int idx = tid; idx < (n - nu) * (ncol - nu); idx += LU_THREADS) {
      int r = nu + idx / (ncol - nu), c = nu + idx % (ncol - nu);
      if (!isfinite(A[(int64_t)r * el.ld + c])) bad = 1;
    }
    bad = __syncthreads_or(bad);
    if (tid == 0 && bad && status[e] == IEDG_ELEM_OK) status[e] = IEDG_ELEM_NONFINITE;
    if (__syncthreads_or(mine.failed)) {
      if (tid == 0) { atomicOr(err, 1); status[e] = IEDG_ELEM_TIMEOUT; }
      tc_drain(mine);     // MMAs still in flight finish before the TMEM is freed
      ++it;
      break;
    }
  }
  if (mine.failed)
    for (; next_element(queue, E, it, lud.order, &e); ++it)
      if (tid == 0) status[e] = IEDG_ELEM_TIMEOUT;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem_base, OZ_TMEM_COLS);
}

}  // namespace

size_t lu64_smem(const Dims& dm, int nb);

template <class T>
static cudaError_t assemble_t(iedg_mesh* M, T* S, const double* rhs64, const AsmTab<T>& tb, cudaStream_t st) {
  const Dims& dm = M->dm;
  AsmCfg cf = asm_cfg(dm);
  const bool mix = M->tt.nb != nullptr;
  int inner = 1;
  for (int r = 0; r < dm.d; ++r) inner *= dm.p - 1;
  const int nbu = dm.Np - inner;                  // boundary nodes of the element
  size_t smem = sizeof(T) * ((size_t)cf.KC * cf.rows_pad + (size_t)cf.KC * cf.CW + (size_t)nbu * cf.CW +
                             (size_t)dm.Nfq * cf.CW + (mix ? (size_t)dm.Nb * cf.CW : 0));
  cudaError_t err = cudaFuncSetAttribute(k_assemble<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  dim3 grid((unsigned)(M->E * dm.m * dm.m), cf.nsplit);
  k_assemble<T><<<grid, AS_THREADS, smem, st>>>(dm, M->ph, cf, M->ref, tb, S, rhs64, M->tt, nbu, nullptr);
  return cudaGetLastError();
}

AsmTab<double> tables64(const iedg_mesh* M) {
  const Geo& G = M->geo;
  const PointJac& P = M->pj;
  return AsmTab<double>{M->ref.Phi, M->ref.Dxi, M->ref.PhiF, P.Jv, P.Jf, P.lamw, P.Su, P.Jb,
                        G.GlV, G.HlV, G.GlF, G.HlF, G.Mass};
}

AsmTab<float> tables32(const iedg_mesh* M) {
  const Geo& G = M->geo;
  const PointJac& P = M->pj;
  return AsmTab<float>{M->ref.Phi32, M->ref.Dxi32, M->ref.PhiF32, P.Jv32, P.Jf32, P.lamw32, P.Su32, P.Jb32,
                       G.GlV32, G.HlV32, G.GlF32, G.HlF32, G.Mass32};
}

cudaError_t launch_assemble_list(iedg_mesh* M, double* S, const int64_t* elist, int64_t n_slots, cudaStream_t st) {
  const Dims& dm = M->dm;
  if (assemble_sf_supported(dm)) return launch_assemble_sf_list(M, S, elist, n_slots, st);
  AsmCfg cf = asm_cfg(dm);
  int inner = 1;
  for (int r = 0; r < dm.d; ++r) inner *= dm.p - 1;
  const int nbu = dm.Np - inner;
  size_t smem = sizeof(double) * ((size_t)cf.KC * cf.rows_pad + (size_t)cf.KC * cf.CW + (size_t)nbu * cf.CW +
                                  (size_t)dm.Nfq * cf.CW);
  cudaError_t err =
      cudaFuncSetAttribute(k_assemble<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  dim3 grid((unsigned)(n_slots * dm.m * dm.m), cf.nsplit);
  k_assemble<double, true><<<grid, AS_THREADS, smem, st>>>(dm, M->ph, cf, M->ref, tables64(M), S, M->rhs64, M->tt,
                                                           nbu, elist);
  return cudaGetLastError();
}

cudaError_t launch_lu64_list(iedg_mesh* M, double* S, int64_t n_slots, const int64_t* active, int8_t* status,
                             cudaStream_t st) {
  const Dims& dm = M->dm;
  size_t smem = lu64_smem(dm, 16);
  cudaError_t err = cudaFuncSetAttribute(k_lu<double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_lu<double, 16><<<(unsigned)n_slots, LU_THREADS, smem, st>>>(dm, LuDesc{}, S, status, nullptr, nullptr, n_slots,
                                                                active);
  return cudaGetLastError();
}

cudaError_t launch_assemble(iedg_mesh* M, cudaStream_t st) {
  if (M->precision == 0) return assemble_t<double>(M, M->S, nullptr, tables64(M), st);
  return assemble_t<float>(M, M->S32, M->rhs64, tables32(M), st);
}

template <class T, int NB>
static cudaError_t lu_t(iedg_mesh* M, T* S, int* piv, cudaStream_t st) {
  const Dims& dm = M->dm;
  size_t smem = sizeof(T) * ((size_t)dm.n * NB + (size_t)NB * UCW);
  cudaError_t err = cudaFuncSetAttribute(k_lu<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (M->sched.lu_persistent) {
    unsigned grid = 0;
    err = persistent_grid(k_lu<T, NB>, smem, M->E, &grid);
    if (err == cudaSuccess) err = cudaMemsetAsync(M->queue, 0, sizeof(int64_t), st);
    if (err != cudaSuccess) return err;
    k_lu<T, NB><<<grid, LU_THREADS, smem, st>>>(dm, M->lud, S, M->status, piv, M->queue, M->E);
  } else {
    k_lu<T, NB><<<(unsigned)M->E, LU_THREADS, smem, st>>>(dm, M->lud, S, M->status, piv, nullptr, M->E);
  }
  return cudaGetLastError();
}

size_t lu64_smem(const Dims& dm, int nb) { return sizeof(double) * ((size_t)dm.n * nb + (size_t)nb * UCW); }

// FP64 form with the Schur complement on the tensor cores (persistent grid only: each
// CTA owns a slice buffer for the element it works on).  The buffers are allocated
// when the schedule selects this form (iedg_set_schedule), never by a compute call.
static cudaError_t lu64_oz_grid(iedg_mesh* M, size_t* smem_out, unsigned* grid, int64_t* per_cta) {
  const Dims& dm = M->dm;
  size_t smem = lu64_smem(dm, 16);
  if (smem < (size_t)OZ_STAGE_BYTES) smem = OZ_STAGE_BYTES;
  cudaError_t err = cudaFuncSetAttribute(k_lu64_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  // two resident CTAs at most: each holds 256 of the SM's 512 TMEM columns
  err = persistent_grid(k_lu64_oz, smem, M->E, grid, 2);
  if (err != cudaSuccess) return err;
  const int64_t ntm = dm.nt + 1;
  *per_cta = ((2 * (int64_t)OZ_S * ntm * dm.nu + 4 * ntm) + 3) & ~(int64_t)3;
  *smem_out = smem;
  return cudaSuccess;
}

cudaError_t prepare_lu64_oz(iedg_mesh* M) {
  size_t smem = 0;
  unsigned grid = 0;
  int64_t per = 0;
  cudaError_t err = lu64_oz_grid(M, &smem, &grid, &per);
  if (err != cudaSuccess) return err;
  if (M->oz_scratch != nullptr && M->oz_grid >= grid) return cudaSuccess;
  if (M->oz_scratch) cudaFree(M->oz_scratch);
  M->oz_scratch = nullptr;
  err = cudaMalloc(&M->oz_scratch, (size_t)grid * per * sizeof(float));
  if (err != cudaSuccess) return err;
  M->oz_grid = grid;
  return cudaSuccess;
}

static cudaError_t lu64_oz(iedg_mesh* M, cudaStream_t st) {
  const Dims& dm = M->dm;
  size_t smem = 0;
  unsigned grid = 0;
  int64_t per = 0;
  cudaError_t err = lu64_oz_grid(M, &smem, &grid, &per);
  if (err != cudaSuccess) return err;
  if (M->oz_scratch == nullptr || M->oz_grid < grid) return cudaErrorNotReady;   // set_schedule allocates
  err = cudaMemsetAsync(M->queue, 0, sizeof(int64_t), st);
  if (err != cudaSuccess) return err;
  k_lu64_oz<<<grid, LU_THREADS, smem, st>>>(dm, M->lud, M->S, M->status, M->queue, M->E, M->oz_scratch, per,
                                             M->dev_flag, tc_wait_limit(M));
  return cudaGetLastError();
}

// FP32 partial LU with the Schur complement on the tensor cores in operand form KIND.
template <int KIND>
static cudaError_t lu32_tc(iedg_mesh* M, cudaStream_t st) {
  const Dims& dm = M->dm;
  // panel + U chunk during the factorisation; the two operand stages of the Schur GEMM
  // reuse the same buffer afterwards
  size_t smem = sizeof(float) * ((size_t)L32_NB * dm.n + (size_t)L32_NB * L32_UCW);
  if (smem < 2 * (size_t)TC_STAGE_BYTES) smem = 2 * (size_t)TC_STAGE_BYTES;
  cudaError_t err = cudaFuncSetAttribute(k_lu32_tc<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  unsigned grid = (unsigned)M->E;
  int64_t* queue = nullptr;
  if (M->sched.lu_persistent) {
    err = persistent_grid(k_lu32_tc<KIND>, smem, M->E, &grid);
    if (err == cudaSuccess) err = cudaMemsetAsync(M->queue, 0, sizeof(int64_t), st);
    if (err != cudaSuccess) return err;
    queue = M->queue;
  }
  k_lu32_tc<KIND><<<grid, LU_THREADS, smem, st>>>(dm, M->lud, M->S32, M->status, M->piv, queue, M->E, M->dev_flag,
                                                   tc_wait_limit(M));
  return cudaGetLastError();
}

cudaError_t launch_lu(iedg_mesh* M, cudaStream_t st) {
  if (M->dm.nu > LU_MAX_NU) return cudaErrorInvalidValue;   // orders above 4 are rejected at creation
  if (M->precision == 0 && M->sched.lu_tensor) return lu64_oz(M, st);
  if (M->precision == 0) {
    if (M->sched.lu_panel == 32 && lu64_smem(M->dm, 32) <= 227 * 1024) return lu_t<double, 32>(M, M->S, nullptr, st);
    return lu_t<double, 16>(M, M->S, nullptr, st);
  }
  if (M->schur_in == kSchurTf32) return lu32_tc<kSchurTf32>(M, st);
  if (M->schur_in == kSchurBf16) return lu32_tc<kSchurBf16>(M, st);
  if (M->sched.lu_tensor == 2) return launch_lu32_mma(M, M->dm.n, st);
  if (M->sched.lu_tensor) return lu32_tc<kSchurFp32>(M, st);
  const Dims& dm = M->dm;
  size_t smem = sizeof(float) * ((size_t)L32_NB * dm.n + (size_t)L32_NB * L32_UCW);
  cudaError_t err = cudaFuncSetAttribute(k_lu32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (M->sched.lu_persistent) {
    unsigned grid = 0;
    err = persistent_grid(k_lu32, smem, M->E, &grid);
    if (err == cudaSuccess) err = cudaMemsetAsync(M->queue, 0, sizeof(int64_t), st);
    if (err != cudaSuccess) return err;
    k_lu32<<<grid, LU_THREADS, smem, st>>>(dm, M->lud, M->S32, M->status, M->piv, M->queue, M->E);
  } else {
    k_lu32<<<(unsigned)M->E, LU_THREADS, smem, st>>>(dm, M->lud, M->S32, M->status, M->piv, nullptr, M->E);
  }
  return cudaGetLastError();
}

}  // namespace iedg
