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
#include "iedg_internal.cuh"

namespace iedg {
namespace {

constexpr int SF_THREADS = 256;
constexpr int SF_CC = 16;          // columns per chunk

template <class T>
size_t sf_smem(const Dims& dm) {
  const int nq1 = dm.nq1, np1 = dm.np1;
  size_t n = 2 * (size_t)nq1 * np1 + 3 * (size_t)dm.Nq * SF_CC + 3 * (size_t)nq1 * nq1 * np1 * SF_CC +
             2 * (size_t)nq1 * np1 * np1 * SF_CC + (size_t)dm.Nb * SF_CC + (size_t)dm.Nfq * SF_CC;
  return n * sizeof(T);
}

// Element sizes are compile-time constants (NP1 = p + 1, NQ1 = p + 2), so every index
// split below is a multiply-shift; every chunk runs over all SF_CC columns with the
// columns past the end masked.
template <class T, int NP1, int NQ1>
__global__ void __launch_bounds__(SF_THREADS)
k_assemble_sf(Dims dm, Phys ph, RefTables ref, AsmTab<T> tb, T* __restrict__ S, const double* __restrict__ rhs64) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int tid = threadIdx.x;
  constexpr int m = 5, m2 = 25, d = 3;
  constexpr int np1 = NP1, nq1 = NQ1;
  constexpr int Np = NP1 * NP1 * NP1, Nq = NQ1 * NQ1 * NQ1, Nfq = NQ1 * NQ1, Nfn = NP1 * NP1;
  constexpr int Nb = Np - (NP1 - 2) * (NP1 - 2) * (NP1 - 2), Nfp = 6 * Nfq;
  const int64_t e = blockIdx.x / m2;
  const int pair = blockIdx.x % m2, i = pair / m, k = pair % m;
  const bool has_cq = !(i == 0 || (i <= d && k == m - 1));
  const int ncol_all = Np + Nb, ncol_vol = has_cq ? Np + Nb : Np;
  T* sL = sm;                                        // [nq1][np1]
  T* sdL = sL + nq1 * np1;                           // [nq1][np1]
  T* W = sdL + nq1 * np1;                            // [3][Nq][CC]
  T* Tt = W + 3 * Nq * SF_CC;                        // [3][nq1 nq1 np1][CC]
  T* V = Tt + 3 * nq1 * nq1 * np1 * SF_CC;           // [2][nq1 np1 np1][CC]
  T* facc = V + 2 * nq1 * np1 * np1 * SF_CC;         // [Nb][CC]
  T* Vf = facc + Nb * SF_CC;                         // [Nfq][CC]
  for (int idx = tid; idx < nq1 * np1; idx += SF_THREADS) { sL[idx] = (T)ref.L1[idx]; sdL[idx] = (T)ref.dL1[idx]; }
  const size_t jvs = (size_t)(1 + d) * d * Nq, jfs = (size_t)(1 + d) * Nfp;
  const T* jv = tb.Jv + ((size_t)e * m2 + pair) * jvs;
  const T* jf = tb.Jf + ((size_t)e * m2 + pair) * jfs;
  const T* GlV = tb.GlV + (size_t)e * d * Nq * Np;
  const T* HlV = tb.HlV + (size_t)e * d * Nq * Nb;
  const T* GlF = tb.GlF + (size_t)e * d * Nfp * Np;
  const T* HlF = tb.HlF + (size_t)e * d * Nfp * Nb;
  const T* Ms = tb.Mass + (size_t)e * Np * Np;
  const T lamsel = (i == k) ? (T)1 : (T)0;
  const T alpha = (T)ph.alpha;
  const int64_t nn = dm.n, ld = dm.ld;
  T* Se = S + e * nn * ld;
  if (rhs64 != nullptr && pair == 0)
    for (int r = tid; r < nn; r += SF_THREADS) Se[r * ld + nn] = (T)rhs64[e * nn + r];
  constexpr int TS = nq1 * nq1 * np1, VS = nq1 * np1 * np1, cw = SF_CC;

  for (int c0 = 0; c0 < ncol_all; c0 += SF_CC) {
    // ---- face parts of the boundary rows for this column chunk
    for (int idx = tid; idx < Nb * SF_CC; idx += SF_THREADS) facc[idx] = (T)0;
    for (int f = 0; f < dm.nf; ++f) {
      __syncthreads();
      for (int idx = tid; idx < Nfq * cw; idx += SF_THREADS) {
        int gf = idx / cw, c = idx % cw, col = c0 + c;
        int fp = f * Nfq + gf;
        T v = 0;
        if (col >= ncol_all) {
        } else if (col < Np) {
          v = lamsel * tb.lamw[e * Nfp + fp] * tb.PhiF[(size_t)fp * Np + col];
          if (has_cq)
            for (int l = 0; l < d; ++l) v -= jf[(size_t)(1 + l) * Nfp + fp] * GlF[((size_t)l * Nfp + fp) * Np + col];
        } else {
          int t = col - Np;
          v = jf[fp] * tb.PhiF[(size_t)fp * Np + ref.bnode[t]];
          if (has_cq)
            for (int l = 0; l < d; ++l) v += jf[(size_t)(1 + l) * Nfp + fp] * HlF[((size_t)l * Nfp + fp) * Nb + t];
        }
        Vf[gf * SF_CC + c] = v;
      }
      __syncthreads();
      for (int idx = tid; idx < Nfn * cw; idx += SF_THREADS) {
        int tn = idx / cw, c = idx % cw;
        int a = ref.fnode[f * Nfn + tn];
        T s = 0;
        for (int gf = 0; gf < Nfq; ++gf) s = fma(tb.PhiF[(size_t)(f * Nfq + gf) * Np + a], Vf[gf * SF_CC + c], s);
        facc[ref.slot[a] * SF_CC + c] += s;
      }
    }
    // ---- volume right operands W_r for this chunk (zero outside the volume columns)
    for (int idx = tid; idx < 3 * Nq * cw; idx += SF_THREADS) {
      int r = idx / (Nq * cw), g = (idx / cw) % Nq, c = idx % cw, col = c0 + c;
      T w = 0;
      if (col < Np) {
        w = jv[(size_t)r * Nq + g] * tb.Phi[(size_t)g * Np + col];
        if (has_cq)
          for (int l = 0; l < d; ++l) w -= jv[(size_t)(d + l * d + r) * Nq + g] * GlV[((size_t)l * Nq + g) * Np + col];
      } else if (col < ncol_vol) {
        for (int l = 0; l < d; ++l)
          w += jv[(size_t)(d + l * d + r) * Nq + g] * HlV[((size_t)l * Nq + g) * Nb + (col - Np)];
      }
      W[(r * Nq + g) * SF_CC + c] = w;
    }
    __syncthreads();
    // stage A: contract g_z.  T_r[gx,gy,az] = sum_gz X_r(gz, az) W_r[gx,gy,gz], X_2 = L', else L
    for (int idx = tid; idx < 3 * TS * cw; idx += SF_THREADS) {
      int r = idx / (TS * cw), t = (idx / cw) % TS, c = idx % cw;
      int gx = t % nq1, gy = (t / nq1) % nq1, az = t / (nq1 * nq1);
      const T* X = r == 2 ? sdL : sL;
      T s = 0;
      for (int gz = 0; gz < nq1; ++gz)
        s = fma(X[gz * np1 + az], W[(r * Nq + gx + nq1 * (gy + nq1 * gz)) * SF_CC + c], s);
      Tt[(r * TS + t) * SF_CC + c] = s;
    }
    __syncthreads();
    // stage B: contract g_y.  V_0 = L_y T_0 (to be contracted with L'_x),
    //                         V_1 = L'_y T_1 + L_y T_2 (to be contracted with L_x)
    for (int idx = tid; idx < VS * cw; idx += SF_THREADS) {
      int t = idx / cw, c = idx % cw;
      int gx = t % nq1, ay = (t / nq1) % np1, az = t / (nq1 * np1);
      T s0 = 0, s1 = 0;
      for (int gy = 0; gy < nq1; ++gy) {
        int tt = gx + nq1 * (gy + nq1 * az);
        T Ly = sL[gy * np1 + ay], dLy = sdL[gy * np1 + ay];
        s0 = fma(Ly, Tt[(0 * TS + tt) * SF_CC + c], s0);
        s1 = fma(dLy, Tt[(1 * TS + tt) * SF_CC + c], s1);
        s1 = fma(Ly, Tt[(2 * TS + tt) * SF_CC + c], s1);
      }
      V[(0 * VS + t) * SF_CC + c] = s0;
      V[(1 * VS + t) * SF_CC + c] = s1;
    }
    __syncthreads();
    // stage C: contract g_x and write the u-rows (volume + faces + mass)
    for (int idx = tid; idx < Np * cw; idx += SF_THREADS) {
      int a = idx / cw, c = idx % cw, col = c0 + c;
      if (col >= ncol_all) continue;
      int ax = a % np1, ay = (a / np1) % np1, az = a / (np1 * np1);
      T s = 0;
      for (int gx = 0; gx < nq1; ++gx) {
        int t = gx + nq1 * (ay + np1 * az);
        s = fma(sdL[gx * np1 + ax], V[(0 * VS + t) * SF_CC + c], s);
        s = fma(sL[gx * np1 + ax], V[(1 * VS + t) * SF_CC + c], s);
      }
      int sl = ref.slot[a];
      if (sl >= 0) s += facc[sl * SF_CC + c];
      if (i == k && col < Np) s += alpha * Ms[a * Np + col];
      int64_t cs = col < Np ? (int64_t)k * Np + col : (int64_t)dm.nu + (int64_t)k * Nb + (col - Np);
      Se[((int64_t)i * Np + a) * ld + cs] = s;
    }
    // trace rows
    for (int idx = tid; idx < Nb * cw; idx += SF_THREADS) {
      int sl = idx / cw, c = idx % cw, col = c0 + c;
      if (col >= ncol_all) continue;
      int64_t cs = col < Np ? (int64_t)k * Np + col : (int64_t)dm.nu + (int64_t)k * Nb + (col - Np);
      Se[((int64_t)dm.nu + (int64_t)i * Nb + sl) * ld + cs] = facc[sl * SF_CC + c];
    }
    __syncthreads();
  }
}

}  // namespace

template <class T, int NP1, int NQ1>
static cudaError_t assemble_sf_t(iedg_mesh* M, T* S, const double* rhs64, const AsmTab<T>& tb, cudaStream_t st) {
  const Dims& dm = M->dm;
  size_t smem = sf_smem<T>(dm);
  auto kern = k_assemble_sf<T, NP1, NQ1>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<(unsigned)(M->E * dm.m * dm.m), SF_THREADS, smem, st>>>(dm, M->ph, M->ref, tb, S, rhs64);
  return cudaGetLastError();
}

template <class T>
static cudaError_t assemble_sf_p(iedg_mesh* M, T* S, const double* rhs64, const AsmTab<T>& tb, cudaStream_t st) {
  switch (M->dm.p) {
    case 2: return assemble_sf_t<T, 3, 4>(M, S, rhs64, tb, st);
    case 3: return assemble_sf_t<T, 4, 5>(M, S, rhs64, tb, st);
    default: return assemble_sf_t<T, 5, 6>(M, S, rhs64, tb, st);
  }
}

bool assemble_sf_supported(const Dims& dm) {
  return dm.d == 3 && dm.p >= 2 && dm.p <= 4 && dm.nq1 == dm.p + 2;
}

cudaError_t launch_assemble_sf(iedg_mesh* M, cudaStream_t st) {
  if (M->precision == 0) return assemble_sf_p<double>(M, M->S, nullptr, tables64(M), st);
  return assemble_sf_p<float>(M, M->S32, M->rhs64, tables32(M), st);
}

}  // namespace iedg
