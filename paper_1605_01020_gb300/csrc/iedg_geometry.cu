// Per-element geometry of the isoparametric map (Sec. 3.1: degree p = k) and the
// element operators of the q-equation (Eq. IEDG a): mass matrix M, lifting
// operators G_l = M^-1 B_l and H_l = M^-1 E_l with
//   B_l[a][b] = sum_g w dphi_a/dx_l phi_b,   E_l[a][t] = sum_fp wf n_l phi_a mu_t,
// and their values at the volume / face quadrature points.  Run once per mesh.
#include "iedg_internal.cuh"

namespace iedg {
namespace {

__device__ inline double cofactor2(const double J[3][3], int i, int r) {
  // cof(J) = detJ J^-T for 2x2
  if (i == 0 && r == 0) return J[1][1];
  if (i == 0 && r == 1) return -J[1][0];
  if (i == 1 && r == 0) return -J[0][1];
  return J[0][0];
}

__device__ inline double cofactor3(const double J[3][3], int i, int r) {
  int i1 = (i + 1) % 3, i2 = (i + 2) % 3, r1 = (r + 1) % 3, r2 = (r + 2) % 3;
  return J[i1][r1] * J[i2][r2] - J[i1][r2] * J[i2][r1];
}

// One CTA per element.
__global__ void k_geometry(Dims dm, RefTables ref, Geo G, const double* __restrict__ X,
                           double* __restrict__ scratch, int* flag, TraceTab tt) {
  extern __shared__ double sm[];
  const int e = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  const int d = dm.d, Np = dm.Np, Nq = dm.Nq, Nb = dm.Nb, Nfp = dm.Nfp, Nfq = dm.Nfq;
  double* sX = sm;                       // [Np][d]
  double* sW = sX + Np * d;              // [Nq]
  double* sJi = sW + Nq;                 // [Nq][d][d]
  double* sfw = sJi + Nq * d * d;        // [Nfp]
  double* sfn = sfw + Nfp;               // [Nfp][d]
  double* sMi = sfn + Nfp * d;           // [Np][Np]  mass matrix, inverted in place
  double* sf = sMi + Np * Np;            // [Np]      Gauss-Jordan column factors
  for (int i = tid; i < Np * d; i += nth) sX[i] = X[(size_t)e * Np * d + i];
  __syncthreads();
  // volume points: J[i][r] = sum_a X[a][i] dphi_r[g][a]
  for (int g = tid; g < Nq; g += nth) {
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < Np; ++a)
      for (int r = 0; r < d; ++r) {
        double dp = ref.Dxi[((size_t)r * Nq + g) * Np + a];
        for (int i = 0; i < d; ++i) J[i][r] += sX[a * d + i] * dp;
      }
    double det = 0;
    if (d == 2) det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    else
      for (int r = 0; r < 3; ++r) det += J[0][r] * cofactor3(J, 0, r);
    if (!(det > 0)) atomicOr(flag, 1);
    double w = ref.Wq[g] * det;
    sW[g] = w;
    G.wdet[(size_t)e * Nq + g] = w;
    for (int r = 0; r < d; ++r)
      for (int i = 0; i < d; ++i) {
        double c = (d == 2 ? cofactor2(J, i, r) : cofactor3(J, i, r)) / det;   // Jinv[r][i]
        sJi[(g * d + r) * d + i] = c;
        G.Jinv[(((size_t)e * Nq + g) * d + r) * d + i] = c;
      }
  }
  // face points: area-scaled normal cof(J) nref, nref = +-e_r
  for (int fp = tid; fp < Nfp; fp += nth) {
    int f = fp / Nfq, rf = f / 2;
    double sgn = (f % 2) ? 1.0 : -1.0;
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < Np; ++a)
      for (int r = 0; r < d; ++r) {
        double dp = ref.DxiF[((size_t)r * Nfp + fp) * Np + a];
        for (int i = 0; i < d; ++i) J[i][r] += sX[a * d + i] * dp;
      }
    double nv[3], mag = 0;
    for (int i = 0; i < d; ++i) {
      nv[i] = sgn * (d == 2 ? cofactor2(J, i, rf) : cofactor3(J, i, rf));
      mag += nv[i] * nv[i];
    }
    mag = sqrt(mag);
    double w = ref.Wf[fp % Nfq] * mag;
    sfw[fp] = w;
    G.fw[(size_t)e * Nfp + fp] = w;
    for (int i = 0; i < d; ++i) {
      sfn[fp * d + i] = nv[i] / mag;
      G.fn[((size_t)e * Nfp + fp) * d + i] = nv[i] / mag;
    }
  }
  __syncthreads();
  // mass matrix
  for (int ab = tid; ab < Np * Np; ab += nth) {
    int a = ab / Np, b = ab % Np;
    double s = 0;
    for (int g = 0; g < Nq; ++g) s += sW[g] * ref.Phi[(size_t)g * Np + a] * ref.Phi[(size_t)g * Np + b];
    sMi[ab] = s;
    G.Mass[(size_t)e * Np * Np + ab] = s;
  }
  // B_l (cols < Np) and E_l (cols >= Np) into scratch [l][a][Np + Nb]
  const int W = Np + Nb;
  double* sc = scratch + (size_t)e * d * Np * W;
  for (int idx = tid; idx < d * Np * W; idx += nth) {
    int l = idx / (Np * W), a = (idx / W) % Np, c = idx % W;
    double s = 0;
    if (c < Np) {
      for (int g = 0; g < Nq; ++g) {
        double gp = 0;
        for (int r = 0; r < d; ++r) gp += ref.Dxi[((size_t)r * Nq + g) * Np + a] * sJi[(g * d + r) * d + l];
        s += sW[g] * gp * ref.Phi[(size_t)g * Np + c];
      }
    } else if (tt.sfl) {
      // mixed orders: the slot's basis on each face it lives on (none for padding slots)
      const int t = c - Np;
      if (t < tt.nb[e]) {
        const int* fl = tt.sfl + ((size_t)e * Nb + t) * 3;
        for (int k = 0; k < 3; ++k) {
          const int code = fl[k];
          if (code < 0) continue;
          const int f = code / tt.NFS, j = code % tt.NFS;
          const double* mu = tt.muf + ((size_t)e * dm.nf + f) * Nfq * tt.NFS + j;
          for (int gf = 0; gf < Nfq; ++gf) {
            const int fp = f * Nfq + gf;
            s += sfw[fp] * sfn[fp * d + l] * ref.PhiF[(size_t)fp * Np + a] * mu[(size_t)gf * tt.NFS];
          }
        }
      }
    } else {
      int bt = ref.bnode[c - Np];
      for (int fp = 0; fp < Nfp; ++fp)
        s += sfw[fp] * sfn[fp * d + l] * ref.PhiF[(size_t)fp * Np + a] * ref.PhiF[(size_t)fp * Np + bt];
    }
    sc[idx] = s;
  }
  __syncthreads();
  // in-place Gauss-Jordan inverse of the SPD mass matrix (no pivoting needed)
  for (int k = 0; k < Np; ++k) {
    for (int i = tid; i < Np; i += nth) sf[i] = sMi[i * Np + k];
    __syncthreads();
    double piv = 1.0 / sf[k];
    for (int j = tid; j < Np; j += nth) sMi[k * Np + j] = (j == k ? 1.0 : sMi[k * Np + j]) * piv;
    __syncthreads();
    for (int ij = tid; ij < Np * Np; ij += nth) {
      int i = ij / Np, j = ij % Np;
      if (i == k) continue;
      sMi[ij] = (j == k ? 0.0 : sMi[ij]) - sf[i] * sMi[k * Np + j];
    }
    __syncthreads();
  }
  // G_l = M^-1 B_l, H_l = M^-1 E_l
  for (int idx = tid; idx < d * Np * W; idx += nth) {
    int l = idx / (Np * W), c = (idx / W) % Np, b = idx % W;
    double s = 0;
    for (int a = 0; a < Np; ++a) s += sMi[c * Np + a] * sc[((size_t)l * Np + a) * W + b];
    if (b < Np) G.Gl[(((size_t)e * d + l) * Np + c) * Np + b] = s;
    else G.Hl[(((size_t)e * d + l) * Np + c) * Nb + (b - Np)] = s;
  }
  __syncthreads();
  // liftings at points: Phi G_l, Phi H_l (volume), PhiF G_l, PhiF H_l (faces)
  const double* Gl = G.Gl + (size_t)e * d * Np * Np;
  const double* Hl = G.Hl + (size_t)e * d * Np * Nb;
  for (int idx = tid; idx < d * (Nq + Nfp) * W; idx += nth) {
    int l = idx / ((Nq + Nfp) * W), g = (idx / W) % (Nq + Nfp), b = idx % W;
    const double* phi = g < Nq ? ref.Phi + (size_t)g * Np : ref.PhiF + (size_t)(g - Nq) * Np;
    double s = 0;
    if (b < Np)
      for (int c = 0; c < Np; ++c) s += phi[c] * Gl[((size_t)l * Np + c) * Np + b];
    else
      for (int c = 0; c < Np; ++c) s += phi[c] * Hl[((size_t)l * Np + c) * Nb + (b - Np)];
    if (g < Nq) {
      if (b < Np) G.GlV[(((size_t)e * d + l) * Nq + g) * Np + b] = s;
      else G.HlV[(((size_t)e * d + l) * Nq + g) * Nb + (b - Np)] = s;
    } else {
      int fp = g - Nq;
      if (b < Np) G.GlF[(((size_t)e * d + l) * Nfp + fp) * Np + b] = s;
      else G.HlF[(((size_t)e * d + l) * Nfp + fp) * Nb + (b - Np)] = s;
    }
  }
}

__global__ void k_to_f32(const double* __restrict__ src, float* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

}  // namespace

cudaError_t launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  k_to_f32<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_geometry(iedg_mesh* M, const double* X, double* scratch, cudaStream_t st) {
  const Dims& dm = M->dm;
  size_t smem = sizeof(double) * ((size_t)dm.Np * dm.d + dm.Nq + (size_t)dm.Nq * dm.d * dm.d + dm.Nfp +
                                  (size_t)dm.Nfp * dm.d + (size_t)dm.Np * dm.Np + dm.Np);
  cudaError_t e = cudaFuncSetAttribute(k_geometry, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_geometry<<<(unsigned)M->E, 256, smem, st>>>(dm, M->ref, M->geo, X, scratch, M->dev_flag, M->tt);
  return cudaGetLastError();
}

}  // namespace iedg
