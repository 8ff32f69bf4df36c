// Element block assembly for hexahedra with sum-factorised volume terms (FP64 for
// the FP64 path, FP32 for the mixed path).
//
// Same element matrix as k_assemble (iedg_assemble.cu): for equation component i
// and unknown component k the u-rows are
//   sum_{g,r} Dxi_r[g][a] W_r[g][col] + face parts + alpha delta_ik M,
// with W_r[g][b] = cu_ikr(g) Phi[g][b] - sum_l cq_iklr(g) Gl_l(g)[b] (and the trace
// columns W_r[g][Np + t] = sum_l cq_iklr(g) Hl_l(g)[t]).  The reference derivative
// tables are tensor products, Dxi_0 = L' (x) L (x) L, Dxi_1 = L (x) L' (x) L,
// Dxi_2 = L (x) L (x) L', so the contraction over the n_q1^3 points is done one
// direction at a time (z, then y, then x): 3340 instead of 24000 multiply-adds per
// column at p = 3.  Pairs (i, k) whose viscous Jacobian vanishes identically (the
// mass equation, and momentum equations with respect to the energy unknown) have no
// volume trace columns and skip the lifted-gradient terms.
//
// Meshes with mixed orders (MIX): the element has n_b,e trace slots and its matrix sits
// at its own offset with its own leading dimension.  The trace basis on a face shared
// with the same order is the element basis there (trace rows = face parts of the
// boundary u-rows restricted to those faces); a face with private nodes of degree q
// has the degree-q Gauss-Lobatto Lagrange basis, contracted in two 1D stages like the
// element basis.
#include "iedg_internal.cuh"
#include "iedg_tc.cuh"

namespace iedg {
namespace {

constexpr int SF_THREADS = 256;

template <class T, int CC>
size_t sf_smem(const Dims& dm, bool mix) {
  const int nq1 = dm.nq1, np1 = dm.np1, d = 3;
  const int nbu = dm.Np - (np1 - 2) * (np1 - 2) * (np1 - 2);
  size_t n = 2 * (size_t)nq1 * np1                                   // L, L'
             + (size_t)(1 + d) * d * dm.Nq + (size_t)(2 + d) * dm.Nfp  // pair coefficients
             + 3 * (size_t)dm.Nq * CC + 3 * (size_t)nq1 * nq1 * np1 * CC + 2 * (size_t)nq1 * np1 * np1 * CC;
  if (!mix && sizeof(T) == 4)   // the six faces' node sums
    n += (size_t)6 * np1 * np1 * CC;
  else                          // facc, Vf, Uf; with mixed orders a wider Uf, tacc and LQ
    n += (size_t)nbu * CC + (size_t)dm.Nfq * CC + (size_t)nq1 * (mix ? 5 : np1) * CC +
         (mix ? (size_t)dm.Nb * CC + 25 * (size_t)nq1 : 0);
  return n * sizeof(T);
}

// Face part of boundary node a for column c from the six faces' node sums fn[f][tn][c]:
// node a = (a0, a1, a2) lies on face 2r where its coordinate r is 0 and on face 2r + 1
// where it is p; its index on that face runs over the two other coordinates in order.
// The faces are summed in increasing order, as the face-by-face accumulation does.
template <class T, int NP1, int CC>
__device__ __forceinline__ T face_sum(const T* fn, int a, int c) {
  const int c3[3] = {a % NP1, (a / NP1) % NP1, a / (NP1 * NP1)};
  T fs = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int r = f >> 1;
    if (c3[r] != ((f & 1) ? NP1 - 1 : 0)) continue;
    const int tn = r == 0 ? c3[1] + NP1 * c3[2] : (r == 1 ? c3[0] + NP1 * c3[2] : c3[0] + NP1 * c3[1]);
    fs += fn[(f * NP1 * NP1 + tn) * CC + c];
  }
  return fs;
}

// Element sizes are compile-time constants (NP1 = p + 1, NQ1 = p + 2), so every index
// split below is a multiply-shift; every chunk runs over all CC columns with the
// columns past the end masked.  The pair's point coefficients are staged in shared
// memory once; each right-operand entry then costs one table load per multiply-add
// group instead of one load per multiply-add.  Face terms are contracted by two 1D
// stages over the face's tangential directions (face point gf = g1 + nq1 g2, face
// node tn = a1 + np1 a2, the face-normal factor of the basis being 1 on the face).
template <class T, int NP1, int NQ1, int CC, bool MIX, bool LIST = false>
__global__ void __launch_bounds__(SF_THREADS)
k_assemble_sf(Dims dm, Phys ph, RefTables ref, AsmTab<T> tb, T* __restrict__ S, const double* __restrict__ rhs64,
              TraceTab tt, const int64_t* __restrict__ elist) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int tid = threadIdx.x;
  constexpr int m = 5, m2 = 25, d = 3;
  constexpr int np1 = NP1, nq1 = NQ1;
  constexpr int Np = NP1 * NP1 * NP1, Nq = NQ1 * NQ1 * NQ1, Nfq = NQ1 * NQ1, Nfn = NP1 * NP1;
  constexpr int NbU = Np - (NP1 - 2) * (NP1 - 2) * (NP1 - 2), Nfp = 6 * Nfq;
  constexpr int TS = nq1 * nq1 * np1, VS = nq1 * np1 * np1, NC = (1 + d) * d;
  constexpr int UW = MIX ? 5 : np1;              // second extent of the face stage buffer
  // FP32 on uniform meshes: the six faces' stages run together (3 barriers per column
  // chunk instead of 18; measured faster in FP32, slower in FP64, whose DFMA pipe is
  // the bound there)
  constexpr bool SIX = !MIX && sizeof(T) == 4;
  // with an element list (FP64 fallback of the mixed path) CTA group `slot` assembles
  // element elist[slot] into matrix slot `slot`
  const int64_t slot = blockIdx.x / m2;
  int64_t e = slot;
  if constexpr (LIST) {
    e = elist[slot];
    if (e < 0) return;
  }
  const int pair = blockIdx.x % m2, i = pair / m, k = pair % m;
  const bool has_cq = !(i == 0 || (i <= d && k == m - 1));
  const int Nb = MIX ? tt.nb[e] : NbU;          // trace slots of this element
  const int NbT = MIX ? dm.Nb : NbU;            // slot stride of the lifting tables
  const int ncol_all = Np + Nb;
  const int ncol_vol = has_cq ? Np + Nb : Np;
  T* sL = sm;                                  // [nq1][np1]
  T* sdL = sL + nq1 * np1;                     // [nq1][np1]
  T* cV = sdL + nq1 * np1;                     // [NC][Nq]   cu_r (c < d), cq_lr (c = d + l d + r)
  T* cF = cV + NC * Nq;                        // [1+d][Nfp] fuh, fq_l
  T* cL = cF + (1 + d) * Nfp;                  // [Nfp]      lambda wf (diagonal pairs)
  T* W = cL + Nfp;                             // [3][Nq][CC]
  T* Tt = W + 3 * Nq * CC;                     // [3][TS][CC]
  T* V = Tt + 3 * TS * CC;                     // [2][VS][CC]
  // face parts of the boundary u-rows (and trace rows): accumulated face by face in
  // facc (tacc), or with SIX the six faces' node sums fn[f][tn][c] formed together
  T* facc = V + 2 * VS * CC;                   // [NbU][CC]
  T* Vf = facc + NbU * CC;                     // [Nfq][CC]
  T* Uf = Vf + Nfq * CC;                       // [nq1 UW][CC]
  T* tacc = MIX ? Uf + nq1 * UW * CC : facc;   // [Nb][CC]   trace rows (MIX), else = facc
  T* sLQ = tacc + (MIX ? dm.Nb * CC : 0);      // [5][nq1][5] (MIX)
  T* fn = V + 2 * VS * CC;                     // [6][Nfn][CC] (SIX)
  for (int idx = tid; idx < nq1 * np1; idx += SF_THREADS) { sL[idx] = (T)ref.L1[idx]; sdL[idx] = (T)ref.dL1[idx]; }
  if (MIX) {
    const T* lq = nullptr;
    if constexpr (sizeof(T) == 8) lq = reinterpret_cast<const T*>(ref.LQ);
    else lq = reinterpret_cast<const T*>(ref.LQ32);
    for (int idx = tid; idx < 25 * nq1; idx += SF_THREADS) sLQ[idx] = lq[idx];
  }
  const T* mutab = nullptr;                    // [nf][Nfq][NFS] of this element (MIX)
  if (MIX) {
    if constexpr (sizeof(T) == 8) mutab = reinterpret_cast<const T*>(tt.muf);
    else mutab = reinterpret_cast<const T*>(tt.muf32);
    mutab += (size_t)e * 6 * Nfq * tt.NFS;
  }
  const size_t jvs = (size_t)NC * Nq, jfs = (size_t)(1 + d) * Nfp;
  const T* jv = tb.Jv + ((size_t)e * m2 + pair) * jvs;
  const T* jf = tb.Jf + ((size_t)e * m2 + pair) * jfs;
  // The pair's point coefficients (two contiguous blocks of the point-Jacobian tables)
  // are staged by one thread with two bulk copies on the TMA engine while the others
  // fill the remaining tables; plain loads where an address is not 16-byte aligned.
  constexpr uint32_t bytesV = NC * Nq * sizeof(T), bytesF = (1 + d) * Nfp * sizeof(T);
  static_assert(bytesV % 16 == 0 && bytesF % 16 == 0 && (2 * nq1 * np1 * sizeof(T)) % 16 == 0,
                "bulk copies need 16-byte sizes and offsets");
  __shared__ __align__(8) uint64_t stage_bar;
  const bool bulk = ((reinterpret_cast<uintptr_t>(jv) | reinterpret_cast<uintptr_t>(jf) |
                      reinterpret_cast<uintptr_t>(cV) | reinterpret_cast<uintptr_t>(cF)) & 15) == 0;
  if (bulk) {
    if (tid == 0) {
      tc::mbar_init(&stage_bar, 1);
      tc::mbar_expect_tx(&stage_bar, bytesV + bytesF);
      tc::bulk_g2s(cV, jv, bytesV, &stage_bar);
      tc::bulk_g2s(cF, jf, bytesF, &stage_bar);
    }
  } else {
    for (int idx = tid; idx < NC * Nq; idx += SF_THREADS) cV[idx] = jv[idx];
    for (int idx = tid; idx < (1 + d) * Nfp; idx += SF_THREADS) cF[idx] = jf[idx];
  }
  // dfhat/du of the pair: lambda wf on the diagonal (Lax-Friedrichs) or wf S_ik (Roe-type)
  for (int idx = tid; idx < Nfp; idx += SF_THREADS)
    cL[idx] = tb.Su ? tb.Su[((size_t)e * m2 + pair) * Nfp + idx] : ((i == k) ? tb.lamw[e * Nfp + idx] : (T)0);
  const T* GlV = tb.GlV + (size_t)e * d * Nq * Np;
  const T* HlV = tb.HlV + (size_t)e * d * Nq * NbT;
  const T* GlF = tb.GlF + (size_t)e * d * Nfp * Np;
  const T* HlF = tb.HlF + (size_t)e * d * Nfp * NbT;
  const T* Ms = tb.Mass + (size_t)e * Np * Np;
  const T alpha = (T)ph.alpha;
  const int64_t nn = MIX ? (int64_t)dm.nu + (int64_t)m * Nb : dm.n;
  const int64_t ld = MIX ? tt.ldv[e] : dm.ld;
  T* Se = MIX ? S + tt.soff[e] : S + (LIST ? slot : e) * nn * ld;
  if (rhs64 != nullptr && pair == 0)
    for (int r = tid; r < nn; r += SF_THREADS) Se[r * ld + nn] = (T)rhs64[e * dm.n + r];
  __syncthreads();     // also publishes the barrier's initialisation
  bool late = false;   // the bulk copies did not complete within the wait limit
  if (bulk) {
    late = !__syncthreads_and(tc::mbar_wait(&stage_bar, 0, kTcWaitLimit));
    if (late) {        // same values by plain loads (a late copy writes the same bytes)
      for (int idx = tid; idx < NC * Nq; idx += SF_THREADS) cV[idx] = jv[idx];
      for (int idx = tid; idx < (1 + d) * Nfp; idx += SF_THREADS) cF[idx] = jf[idx];
      __syncthreads();
    }
  }

  for (int c0 = 0; c0 < ncol_all; c0 += CC) {
    // ---- face parts of the boundary rows for this column chunk
    if constexpr (SIX) {
      // all six faces per phase: right operand at the face points, then the two 1D
      // stages; the first two live in the volume buffer W, free until the volume stage
      T* Vf6 = W;                              // [6][Nfq][CC]
      T* Uf6 = W + 6 * Nfq * CC;               // [6][nq1][np1][CC]
      static_assert(6 * (Nfq + nq1 * np1) <= 3 * Nq, "face stages must fit the volume buffer");
      for (int idx = tid; idx < 6 * Nfq * CC; idx += SF_THREADS) {
        const int fp = idx / CC, c = idx % CC, col = c0 + c;
        T v = 0;
        if (col < Np) {
          v = cL[fp] * tb.PhiF[(size_t)fp * Np + col];
          if (has_cq)
            for (int l = 0; l < d; ++l) v -= cF[(1 + l) * Nfp + fp] * GlF[((size_t)l * Nfp + fp) * Np + col];
        } else if (col < ncol_all) {
          const int t = col - Np;
          v = cF[fp] * tb.PhiF[(size_t)fp * Np + ref.bnode[t]];
          if (has_cq)
            for (int l = 0; l < d; ++l) v += cF[(1 + l) * Nfp + fp] * HlF[((size_t)l * Nfp + fp) * NbT + t];
        }
        Vf6[idx] = v;
      }
      __syncthreads();
      // U[f][g1][a2] = sum_g2 L[g2][a2] Vf[f][g1 + nq1 g2]
      for (int idx = tid; idx < 6 * nq1 * np1 * CC; idx += SF_THREADS) {
        const int c = idx % CC, t = idx / CC, f = t / (nq1 * np1), g1 = (t / np1) % nq1, a2 = t % np1;
        T u = 0;
        for (int g2 = 0; g2 < nq1; ++g2) u = fma(sL[g2 * np1 + a2], Vf6[(f * Nfq + g1 + nq1 * g2) * CC + c], u);
        Uf6[idx] = u;
      }
      __syncthreads();
      // node (a1, a2) of face f: sum_g1 L[g1][a1] U[f][g1][a2]
      for (int idx = tid; idx < 6 * Nfn * CC; idx += SF_THREADS) {
        const int c = idx % CC, t = idx / CC, f = t / Nfn, tn = t % Nfn, a1 = tn % np1, a2 = tn / np1;
        T sacc = 0;
        for (int g1 = 0; g1 < nq1; ++g1)
          sacc = fma(sL[g1 * np1 + a1], Uf6[((f * nq1 + g1) * np1 + a2) * CC + c], sacc);
        fn[idx] = sacc;
      }
      __syncthreads();
    }
    if constexpr (!SIX) {
    for (int idx = tid; idx < NbU * CC; idx += SF_THREADS) facc[idx] = (T)0;
    if (MIX)
      for (int idx = tid; idx < Nb * CC; idx += SF_THREADS) tacc[idx] = (T)0;
    for (int f = 0; f < 6; ++f) {
      const int fq = MIX ? tt.fdeg[e * 6 + f] : 0;
      const int* fsf = MIX ? tt.fs + ((size_t)e * 6 + f) * tt.NFS : nullptr;
      __syncthreads();
      for (int idx = tid; idx < Nfq * CC; idx += SF_THREADS) {
        const int gf = idx / CC, c = idx % CC, col = c0 + c;
        const int fp = f * Nfq + gf;
        T v = 0;
        if (col < Np) {
          v = cL[fp] * tb.PhiF[(size_t)fp * Np + col];
          if (has_cq)
            for (int l = 0; l < d; ++l) v -= cF[(1 + l) * Nfp + fp] * GlF[((size_t)l * Nfp + fp) * Np + col];
        } else if (col < ncol_all) {
          const int t = col - Np;
          T mu = 0;
          if (MIX) {
            const int* fl = tt.sfl + ((size_t)e * dm.Nb + t) * 3;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              const int code = fl[q];
              if (code >= 0 && code / tt.NFS == f) mu = mutab[((size_t)f * Nfq + gf) * tt.NFS + code % tt.NFS];
            }
          } else {
            mu = tb.PhiF[(size_t)fp * Np + ref.bnode[t]];
          }
          v = cF[fp] * mu;
          if (has_cq)
            for (int l = 0; l < d; ++l) v += cF[(1 + l) * Nfp + fp] * HlF[((size_t)l * Nfp + fp) * NbT + t];
        }
        Vf[gf * CC + c] = v;
      }
      __syncthreads();
      // U[g1][a2] = sum_g2 L[g2][a2] Vf[g1 + nq1 g2]
      for (int idx = tid; idx < nq1 * np1 * CC; idx += SF_THREADS) {
        const int t = idx / CC, c = idx % CC, g1 = t % nq1, a2 = t / nq1;
        T u = 0;
        for (int g2 = 0; g2 < nq1; ++g2) u = fma(sL[g2 * np1 + a2], Vf[(g1 + nq1 * g2) * CC + c], u);
        Uf[(g1 * UW + a2) * CC + c] = u;
      }
      __syncthreads();
      // node (a1, a2) of the face: sum_g1 L[g1][a1] U[g1][a2]
      for (int idx = tid; idx < Nfn * CC; idx += SF_THREADS) {
        const int tn = idx / CC, c = idx % CC, a1 = tn % np1, a2 = tn / np1;
        T s = 0;
        for (int g1 = 0; g1 < nq1; ++g1) s = fma(sL[g1 * np1 + a1], Uf[(g1 * UW + a2) * CC + c], s);
        facc[ref.slot[ref.fnode[f * Nfn + tn]] * CC + c] += s;
        if (MIX && fq == 0) tacc[fsf[tn] * CC + c] += s;   // continuous face: same sums, trace rows
      }
      if (MIX && fq > 0) {
        __syncthreads();
        if (tt.fkind && tt.fkind[e * 6 + f] != kFaceInterior) {
          // domain-boundary face: the trace rows take the boundary flux; rebuild the
          // right operand from its derivatives (wf dbhat/duhat, dbhat/du, dbhat/dq_l)
          const T* jbt = tb.Jb;
          for (int idx = tid; idx < Nfq * CC; idx += SF_THREADS) {
            const int gf = idx / CC, c = idx % CC, col = c0 + c;
            const int fp = f * Nfq + gf;
            const T* jb = jbt + ((size_t)e * m2 + pair) * (2 + d) * Nfp + fp;
            T v = 0;
            if (col < Np) {
              v = jb[(size_t)Nfp] * tb.PhiF[(size_t)fp * Np + col];
              for (int l = 0; l < d; ++l) v -= jb[(size_t)(2 + l) * Nfp] * GlF[((size_t)l * Nfp + fp) * Np + col];
            } else if (col < ncol_all) {
              const int t = col - Np;
              T mu = 0;
              const int* fl = tt.sfl + ((size_t)e * dm.Nb + t) * 3;
#pragma unroll
              for (int q = 0; q < 3; ++q) {
                const int code = fl[q];
                if (code >= 0 && code / tt.NFS == f) mu = mutab[((size_t)f * Nfq + gf) * tt.NFS + code % tt.NFS];
              }
              v = jb[0] * mu;
              for (int l = 0; l < d; ++l) v += jb[(size_t)(2 + l) * Nfp] * HlF[((size_t)l * Nfp + fp) * NbT + t];
            }
            Vf[gf * CC + c] = v;
          }
          __syncthreads();
        }
        // trace rows of the face's private nodes j = j1 + (q+1) j2:
        // sum_{g1,g2} LQ_q[g1][j1] LQ_q[g2][j2] Vf[g1 + nq1 g2]
        const int q1 = fq + 1;
        const T* Lq = sLQ + fq * nq1 * 5;
        for (int idx = tid; idx < nq1 * q1 * CC; idx += SF_THREADS) {
          const int t = idx / CC, c = idx % CC, g1 = t % nq1, j2 = t / nq1;
          T u = 0;
          for (int g2 = 0; g2 < nq1; ++g2) u = fma(Lq[g2 * 5 + j2], Vf[(g1 + nq1 * g2) * CC + c], u);
          Uf[(g1 * UW + j2) * CC + c] = u;
        }
        __syncthreads();
        for (int idx = tid; idx < q1 * q1 * CC; idx += SF_THREADS) {
          const int j = idx / CC, c = idx % CC, j1 = j % q1, j2 = j / q1;
          T s = 0;
          for (int g1 = 0; g1 < nq1; ++g1) s = fma(Lq[g1 * 5 + j1], Uf[(g1 * UW + j2) * CC + c], s);
          tacc[fsf[j] * CC + c] += s;
        }
        __syncthreads();
      }
    }
    }
    // ---- volume right operands W_r[g][c] for the three reference directions.  The
    // table values of all of this thread's (g, c) entries are requested first, then
    // combined, so their latencies overlap instead of adding up.
    {
      constexpr int WPT = (Nq * CC + SF_THREADS - 1) / SF_THREADS;
      T lv[WPT][4];
#pragma unroll
      for (int u = 0; u < WPT; ++u) {
        const int idx = tid + u * SF_THREADS, g = idx / CC, c = idx % CC, col = c0 + c;
        lv[u][0] = lv[u][1] = lv[u][2] = lv[u][3] = 0;
        if (idx < Nq * CC) {
          if (col < Np) {
            lv[u][0] = tb.Phi[(size_t)g * Np + col];
            if (has_cq)
#pragma unroll
              for (int l = 0; l < d; ++l) lv[u][1 + l] = GlV[((size_t)l * Nq + g) * Np + col];
          } else if (col < ncol_vol) {
#pragma unroll
            for (int l = 0; l < d; ++l) lv[u][1 + l] = HlV[((size_t)l * Nq + g) * NbT + (col - Np)];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < WPT; ++u) {
        const int idx = tid + u * SF_THREADS, g = idx / CC, c = idx % CC, col = c0 + c;
        if (idx >= Nq * CC) break;
        T w0 = 0, w1 = 0, w2 = 0;
        if (col < Np) {
          const T ph_ = lv[u][0];
          w0 = cV[0 * Nq + g] * ph_;
          w1 = cV[1 * Nq + g] * ph_;
          w2 = cV[2 * Nq + g] * ph_;
          if (has_cq)
#pragma unroll
            for (int l = 0; l < d; ++l) {
              const T gv = lv[u][1 + l];
              w0 -= cV[(d + l * d + 0) * Nq + g] * gv;
              w1 -= cV[(d + l * d + 1) * Nq + g] * gv;
              w2 -= cV[(d + l * d + 2) * Nq + g] * gv;
            }
        } else if (col < ncol_vol) {
#pragma unroll
          for (int l = 0; l < d; ++l) {
            const T hv = lv[u][1 + l];
            w0 += cV[(d + l * d + 0) * Nq + g] * hv;
            w1 += cV[(d + l * d + 1) * Nq + g] * hv;
            w2 += cV[(d + l * d + 2) * Nq + g] * hv;
          }
        }
        W[(0 * Nq + g) * CC + c] = w0;
        W[(1 * Nq + g) * CC + c] = w1;
        W[(2 * Nq + g) * CC + c] = w2;
      }
    }
    __syncthreads();
    // stage A: contract g_z.  T_r[gx,gy,az] = sum_gz X_r(gz, az) W_r[gx,gy,gz], X_2 = L', else L
    for (int idx = tid; idx < 3 * TS * CC; idx += SF_THREADS) {
      const int r = idx / (TS * CC), t = (idx / CC) % TS, c = idx % CC;
      const int gxy = t % (nq1 * nq1), az = t / (nq1 * nq1);
      const T* X = r == 2 ? sdL : sL;
      T s = 0;
      for (int gz = 0; gz < nq1; ++gz) s = fma(X[gz * np1 + az], W[(r * Nq + gxy + nq1 * nq1 * gz) * CC + c], s);
      Tt[(r * TS + t) * CC + c] = s;
    }
    __syncthreads();
    // stage B: contract g_y.  V_0 = L_y T_0 (to be contracted with L'_x),
    //                         V_1 = L'_y T_1 + L_y T_2 (to be contracted with L_x)
    for (int idx = tid; idx < VS * CC; idx += SF_THREADS) {
      const int t = idx / CC, c = idx % CC;
      const int gx = t % nq1, ay = (t / nq1) % np1, az = t / (nq1 * np1);
      T s0 = 0, s1 = 0;
      for (int gy = 0; gy < nq1; ++gy) {
        const int tt = gx + nq1 * (gy + nq1 * az);
        const T Ly = sL[gy * np1 + ay], dLy = sdL[gy * np1 + ay];
        s0 = fma(Ly, Tt[(0 * TS + tt) * CC + c], s0);
        s1 = fma(dLy, Tt[(1 * TS + tt) * CC + c], s1);
        s1 = fma(Ly, Tt[(2 * TS + tt) * CC + c], s1);
      }
      V[(0 * VS + t) * CC + c] = s0;
      V[(1 * VS + t) * CC + c] = s1;
    }
    __syncthreads();
    // stage C: contract g_x and write the u-rows (volume + faces + mass)
    for (int idx = tid; idx < Np * CC; idx += SF_THREADS) {
      const int a = idx / CC, c = idx % CC, col = c0 + c;
      if (col >= ncol_all) continue;
      const int ax = a % np1, ayz = a / np1;
      T s = 0;
      for (int gx = 0; gx < nq1; ++gx) {
        const int t = gx + nq1 * ayz;
        s = fma(sdL[gx * np1 + ax], V[(0 * VS + t) * CC + c], s);
        s = fma(sL[gx * np1 + ax], V[(1 * VS + t) * CC + c], s);
      }
      const int sl = ref.slot[a];
      if (sl >= 0) s += SIX ? face_sum<T, NP1, CC>(fn, a, c) : facc[sl * CC + c];
      if (i == k && col < Np) s += alpha * Ms[a * Np + col];
      const int64_t cs = col < Np ? (int64_t)k * Np + col : (int64_t)dm.nu + (int64_t)k * Nb + (col - Np);
      Se[((int64_t)i * Np + a) * ld + cs] = s;
    }
    // trace rows
    for (int idx = tid; idx < Nb * CC; idx += SF_THREADS) {
      const int sl = idx / CC, c = idx % CC, col = c0 + c;
      if (col >= ncol_all) continue;
      const int64_t cs = col < Np ? (int64_t)k * Np + col : (int64_t)dm.nu + (int64_t)k * Nb + (col - Np);
      Se[((int64_t)dm.nu + (int64_t)i * Nb + sl) * ld + cs] =
          SIX ? face_sum<T, NP1, CC>(fn, ref.bnode[sl], c) : tacc[sl * CC + c];
    }
    __syncthreads();
  }
  if (late && tid == 0) tc::mbar_wait(&stage_bar, 0, kTcWaitLimit);   // no copy in flight at exit
}

}  // namespace

template <class T, int NP1, int NQ1, int CC>
static cudaError_t assemble_sf_t(iedg_mesh* M, T* S, const double* rhs64, const AsmTab<T>& tb, cudaStream_t st,
                                 const int64_t* elist, int64_t n_slots) {
  const Dims& dm = M->dm;
  const bool mix = M->tt.nb != nullptr;
  size_t smem = sf_smem<T, CC>(dm, mix);
  auto kern = elist ? k_assemble_sf<T, NP1, NQ1, CC, false, true>
                    : (mix ? k_assemble_sf<T, NP1, NQ1, CC, true> : k_assemble_sf<T, NP1, NQ1, CC, false>);
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int64_t E = elist ? n_slots : M->E;
  kern<<<(unsigned)(E * dm.m * dm.m), SF_THREADS, smem, st>>>(dm, M->ph, M->ref, tb, S, rhs64, M->tt, elist);
  return cudaGetLastError();
}

// column chunk: the schedule's choice (8, 16 or 32 columns), default 8 for FP64
// (more CTAs per SM) and 16 for FP32; a chunk whose shared memory does not fit
// falls back to 8
template <class T, int NP1, int NQ1>
static cudaError_t assemble_sf_c(iedg_mesh* M, T* S, const double* rhs64, const AsmTab<T>& tb, cudaStream_t st,
                                 const int64_t* elist, int64_t n_slots) {
  int cc = M->sched.asm_chunk ? M->sched.asm_chunk : (sizeof(T) == 8 ? 8 : 16);
  if (sizeof(T) == 8 && M->precision != 0) cc = 8;   // FP64 fallback of a mixed handle: the FP64 default
  const bool mix = M->tt.nb != nullptr;
  if (cc == 32 && sf_smem<T, 32>(M->dm, mix) > 227 * 1024) cc = 16;
  if (cc == 16 && sf_smem<T, 16>(M->dm, mix) > 227 * 1024) cc = 8;
  if (cc == 32) return assemble_sf_t<T, NP1, NQ1, 32>(M, S, rhs64, tb, st, elist, n_slots);
  if (cc == 16) return assemble_sf_t<T, NP1, NQ1, 16>(M, S, rhs64, tb, st, elist, n_slots);
  return assemble_sf_t<T, NP1, NQ1, 8>(M, S, rhs64, tb, st, elist, n_slots);
}

template <class T>
static cudaError_t assemble_sf_p(iedg_mesh* M, T* S, const double* rhs64, const AsmTab<T>& tb, cudaStream_t st,
                                 const int64_t* elist = nullptr, int64_t n_slots = 0) {
  switch (M->dm.p) {
    case 2: return assemble_sf_c<T, 3, 4>(M, S, rhs64, tb, st, elist, n_slots);
    case 3: return assemble_sf_c<T, 4, 5>(M, S, rhs64, tb, st, elist, n_slots);
    default: return assemble_sf_c<T, 5, 6>(M, S, rhs64, tb, st, elist, n_slots);
  }
}

bool assemble_sf_supported(const Dims& dm) {
  return dm.d == 3 && dm.p >= 2 && dm.p <= 4 && dm.nq1 == dm.p + 2;
}

cudaError_t launch_assemble_sf(iedg_mesh* M, cudaStream_t st) {
  if (M->precision == 0) return assemble_sf_p<double>(M, M->S, nullptr, tables64(M), st);
  return assemble_sf_p<float>(M, M->S32, M->rhs64, tables32(M), st);
}

cudaError_t launch_assemble_sf_list(iedg_mesh* M, double* S, const int64_t* elist, int64_t n_slots, cudaStream_t st) {
  return assemble_sf_p<double>(M, S, M->rhs64, tables64(M), st, elist, n_slots);
}

}  // namespace iedg
