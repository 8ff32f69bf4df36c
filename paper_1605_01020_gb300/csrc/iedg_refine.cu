// Mixed-precision condensation: FP64 iterative refinement on top of the FP32
// partial LU of the bordered element matrix.
//
// The FP32 factors give K_e to FP32 accuracy (times the conditioning of A~).  The
// right-hand side R_e = G~ - C~ A~^-1 F~ and the element updates
// du = A~^-1 (F~ - B~ dU) are recovered to FP64 accuracy by iterative refinement:
//   x <- LU32^-1 b;  repeat  r = b - A~ x (FP64),  x <- x + LU32^-1 r
// where A~ x, B~ z, C~ x are applied matrix-free in FP64 from the point Jacobians
// and the lifted operators (the same element operator the assembly kernel forms,
// see iedg_assemble.cu), so no FP64 element matrix is ever built.
#include "iedg_internal.cuh"

namespace iedg {
namespace {

constexpr int RF_THREADS = 512;
constexpr int RF_NB = 32;            // panel width of the FP32 factorisation (k_lu<float, 32>)

// The solves stage rows of the FP32 factors in shared memory: one slot of RF_SLOT floats
// (32 used; the stride keeps 16-byte reads of 8 consecutive slots on distinct banks) per
// thread that holds a row, threads 0 .. min(RF_THREADS, nu + 32) - 1.  The slots live in
// the element operator's work arrays dqn .. tbf, free while a solve runs; stage_pad
// pads that region where it is smaller (two doubles of slack for the 16-byte alignment).
constexpr int RF_SLOT = 36;

__host__ __device__ inline int stage_doubles(const Dims& dm) {
  const int slots = dm.nu + 32 < RF_THREADS ? dm.nu + 32 : RF_THREADS;
  return slots * (RF_SLOT / 2) + 2;
}
__host__ __device__ inline int stage_pad(const Dims& dm) {
  const int m = dm.m, d = dm.d;
  const int region = m * d * dm.Np + m * dm.Nq * (1 + 2 * d) + m * dm.Nfp * (4 + d);
  return stage_doubles(dm) > region ? stage_doubles(dm) - region : 0;
}

struct Work {
  double *x, *z, *v, *b, *dqn, *xv, *xq, *tv, *xf, *zf, *xqf, *tf, *tbf, *ou, *ot, *red;
  double *sL, *sdL;              // 1D tables (3D sum factorisation)
};

__device__ Work carve(const Dims& dm, double* sm) {
  Work w;
  const int m = dm.m, d = dm.d;
  double* p = sm;
  w.x = p;   p += dm.nu;
  w.z = p;   p += dm.nt;
  w.v = p;   p += dm.nu;
  w.b = p;   p += dm.nu;
  w.dqn = p; p += m * d * dm.Np;
  w.xv = p;  p += m * dm.Nq;
  w.xq = p;  p += m * d * dm.Nq;
  w.tv = p;  p += m * d * dm.Nq;
  w.xf = p;  p += m * dm.Nfp;
  w.zf = p;  p += m * dm.Nfp;
  w.xqf = p; p += m * d * dm.Nfp;
  w.tf = p;  p += m * dm.Nfp;
  w.tbf = p; p += m * dm.Nfp;
  p += stage_pad(dm);
  w.ou = p;  p += dm.nu;
  w.ot = p;  p += dm.nt;
  w.red = p; p += 32;
  w.sL = p;  p += dm.nq1 * dm.np1;
  w.sdL = p; p += dm.nq1 * dm.np1;
  return w;
}

// the solves' staging slots: dqn rounded up to 16 bytes
__device__ __forceinline__ float* stage_ptr(const Work& w) {
  return reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(w.dqn) + 15) & ~static_cast<uintptr_t>(15));
}

size_t work_doubles(const Dims& dm) {
  const int m = dm.m, d = dm.d;
  return (size_t)3 * dm.nu + dm.nt + (size_t)m * d * dm.Np + (size_t)m * dm.Nq * (1 + 2 * d) +
         (size_t)m * dm.Nfp * (4 + d) + stage_pad(dm) + dm.nu + dm.nt + 32 + 2 * (size_t)dm.nq1 * dm.np1;
}

__device__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < RF_THREADS / 32; ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

// Face part of the u-row of boundary node a, component i, from the face projections
// fb[i][f][tn] (3D): node a lies on face 2r where its coordinate r is 0 and on face
// 2r + 1 where it is p, at index tn over its two other coordinates in order.
__device__ __forceinline__ double face_part(const Dims& dm, const double* fb, int i, int a) {
  const int np1 = dm.np1, Nfn1 = np1 * np1;
  const int c3[3] = {a % np1, (a / np1) % np1, a / (np1 * np1)};
  double s = 0.0;
  for (int f = 0; f < 6; ++f) {
    const int r = f >> 1;
    if (c3[r] != ((f & 1) ? np1 - 1 : 0)) continue;
    const int tn = r == 0 ? c3[1] + np1 * c3[2] : (r == 1 ? c3[0] + np1 * c3[2] : c3[0] + np1 * c3[1]);
    s += fb[((size_t)i * 6 + f) * Nfn1 + tn];
  }
  return s;
}

// ou = A~ x + B~ z (u-rows), ot = C~ x + D~ z (trace rows), all FP64.
// use_x / use_z = false skip the terms of an operand that is identically zero.
// z and ot are component-major with slot stride Nb = Dims.Nb; with mixed orders only
// the element's first nb slots are used (the rest stay zero).
__device__ void element_apply(const Dims& dm, const Phys& ph, const RefTables& ref, const Geo& G,
                              const PointJac& PJ, const TraceTab& tt, int64_t e, Work& w, bool use_x,
                              bool use_z) {
  const int tid = threadIdx.x;
  const int m = dm.m, d = dm.d, Np = dm.Np, Nb = dm.Nb, Nq = dm.Nq, Nfp = dm.Nfp, Nfq = dm.Nfq;
  const int Nfn = dm.Nfn;
  const int nbe = tt.nb ? tt.nb[e] : Nb;
  // nodal lifted gradient of (x, z): dq_kl = -G_l x_k + H_l z_k.  One thread per row
  // (l, c) of G_l | H_l for all m components: each row is read once and no partial
  // sums need combining (FP64 adds are as slow as FP64 FMAs here).
  for (int row = tid; row < d * Np; row += RF_THREADS) {
    const int l = row / Np, c = row % Np;
    const double* gl = G.Gl + (((size_t)e * d + l) * Np + c) * Np;
    const double* hl = G.Hl + (((size_t)e * d + l) * Np + c) * Nb;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (use_x)
      for (int b = 0; b < Np; ++b) {
        const double g = gl[b];
#pragma unroll
        for (int k = 0; k < 5; ++k)
          if (k < m) acc[k] = fma(-g, w.x[k * Np + b], acc[k]);
      }
    if (use_z)
      for (int t = 0; t < nbe; ++t) {
        const double h = hl[t];
#pragma unroll
        for (int k = 0; k < 5; ++k)
          if (k < m) acc[k] = fma(h, w.z[k * Nb + t], acc[k]);
      }
#pragma unroll
    for (int k = 0; k < 5; ++k)
      if (k < m) w.dqn[(k * d + l) * Np + c] = acc[k];
  }
  __syncthreads();
  // values at volume points (rows: x_k, then dq_kl)
  const int nrow = m + m * d;
  if (d == 3) {
    // tensor-product interpolation, one direction at a time: x, then y, into the
    // region tv | xf | zf | xqf (contiguous in the work layout; tv is free here and the
    // face values are written only later; nrow (S1 + S2) fits it for p <= 4 and every
    // quad_extra), then z into the point values
    const int np1 = dm.np1, nq1 = dm.nq1;
    const int S1 = nq1 * np1 * np1, S2 = nq1 * nq1 * np1;
    double* t1 = w.tv;
    double* t2 = w.tv + (size_t)nrow * S1;
    for (int idx = tid; idx < nrow * S1; idx += RF_THREADS) {
      int row = idx / S1, t = idx % S1;
      int gx = t % nq1, ayz = t / nq1;
      const double* src = (row < m ? w.x + row * Np : w.dqn + (row - m) * Np) + np1 * ayz;
      double s = 0.0;
      for (int ax = 0; ax < np1; ++ax) s = fma(w.sL[gx * np1 + ax], src[ax], s);
      t1[idx] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < nrow * S2; idx += RF_THREADS) {
      int row = idx / S2, t = idx % S2;
      int gx = t % nq1, gy = (t / nq1) % nq1, az = t / (nq1 * nq1);
      const double* src = t1 + row * S1 + gx + nq1 * np1 * az;
      double s = 0.0;
      for (int ay = 0; ay < np1; ++ay) s = fma(w.sL[gy * np1 + ay], src[nq1 * ay], s);
      t2[idx] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < nrow * Nq; idx += RF_THREADS) {
      int row = idx / Nq, g = idx % Nq;
      int gxy = g % (nq1 * nq1), gz = g / (nq1 * nq1);
      const double* src = t2 + row * S2 + gxy;
      double s = 0.0;
      for (int az = 0; az < np1; ++az) s = fma(w.sL[gz * np1 + az], src[nq1 * nq1 * az], s);
      if (row < m) w.xv[row * Nq + g] = s;
      else w.xq[(row - m) * Nq + g] = s;
    }
    __syncthreads();
    // values of x (if used) and dq at the face points: on face f the face nodes form
    // an np1 x np1 lattice over the two tangential directions (in the order of fnode)
    // and the face points an nq1 x nq1 lattice, so two 1D stages per face
    const int xr = use_x ? m : 0, nr = xr + m * d, nf = dm.nf;
    const int FA = nq1 * np1;
    double* u1 = w.tv;                      // rows in chunks of rc: rc * nf * FA <= m d Nq
    const int rc = (m * d * Nq) / (nf * FA);
    for (int r0 = 0; r0 < nr; r0 += rc) {
      const int r1 = min(nr, r0 + rc);
      for (int idx = tid; idx < (r1 - r0) * nf * FA; idx += RF_THREADS) {
        int row = r0 + idx / (nf * FA), f = (idx / FA) % nf, t = idx % FA;
        int g0 = t % nq1, a1 = t / nq1;
        const int* fn = ref.fnode + f * Nfn + np1 * a1;
        const double* src = row < xr ? w.x + row * Np : w.dqn + (row - xr) * Np;
        double s = 0.0;
        for (int a0 = 0; a0 < np1; ++a0) s = fma(w.sL[g0 * np1 + a0], src[fn[a0]], s);
        u1[idx] = s;
      }
      __syncthreads();
      for (int idx = tid; idx < (r1 - r0) * Nfp; idx += RF_THREADS) {
        int row = r0 + idx / Nfp, fp = idx % Nfp, f = fp / Nfq, gf = fp % Nfq;
        int g0 = gf % nq1, g1 = gf / nq1;
        const double* src = u1 + ((size_t)(row - r0) * nf + f) * FA + g0;
        double s = 0.0;
        for (int a1 = 0; a1 < np1; ++a1) s = fma(w.sL[g1 * np1 + a1], src[nq1 * a1], s);
        if (row < xr) w.xf[row * Nfp + fp] = s;
        else w.xqf[(row - xr) * Nfp + fp] = s;
      }
      __syncthreads();
    }
  } else {
    for (int idx = tid; idx < nrow * Nq; idx += RF_THREADS) {
      int row = idx / Nq, g = idx % Nq;
      const double* src = row < m ? w.x + row * Np : w.dqn + (row - m) * Np;
      const double* phi = ref.Phi + (size_t)g * Np;
      double s = 0.0;
      for (int c = 0; c < Np; ++c) s = fma(phi[c], src[c], s);
      if (row < m) w.xv[row * Nq + g] = s;
      else w.xq[(row - m) * Nq + g] = s;
    }
  }
  // values at face points from the face nodes: every row in 2D, the trace rows in 3D
  for (int idx = tid; idx < (2 * m + m * d) * Nfp; idx += RF_THREADS) {
    int row = idx / Nfp, fp = idx % Nfp, f = fp / Nfq;
    if ((row < m && !use_x) || (row >= m && row < 2 * m && !use_z)) continue;
    if (d == 3 && (row < m || row >= 2 * m)) continue;
    const double* phi = ref.PhiF + (size_t)fp * Np;
    double s = 0.0;
    if (tt.nfs && row >= m && row < 2 * m) {
      // trace basis of this face from the element's table
      const int cnt = tt.nfs[e * dm.nf + f];
      const int* fsf = tt.fs + ((size_t)e * dm.nf + f) * tt.NFS;
      const double* mu = tt.muf + (((size_t)e * dm.nf + f) * Nfq + (fp - f * Nfq)) * tt.NFS;
      for (int j = 0; j < cnt; ++j) s = fma(mu[j], w.z[(row - m) * Nb + fsf[j]], s);
    } else
    for (int tn = 0; tn < Nfn; ++tn) {
      int a = ref.fnode[f * Nfn + tn];
      double v;
      if (row < m) v = w.x[row * Np + a];
      else if (row < 2 * m) v = w.z[(row - m) * Nb + ref.slot[a]];
      else v = w.dqn[(row - 2 * m) * Np + a];
      s = fma(phi[a], v, s);
    }
    if (row < m) w.xf[row * Nfp + fp] = s;
    else if (row < 2 * m) w.zf[(row - m) * Nfp + fp] = s;
    else w.xqf[(row - 2 * m) * Nfp + fp] = s;
  }
  __syncthreads();
  // pointwise linearised fluxes (weights and Jinv already folded in the tables)
  const size_t jvs = (size_t)(1 + d) * d * Nq, jfs = (size_t)(1 + d) * Nfp;
  const double* jv = PJ.Jv + (size_t)e * m * m * jvs;
  const double* jf = PJ.Jf + (size_t)e * m * m * jfs;
  for (int idx = tid; idx < m * d * Nq; idx += RF_THREADS) {
    int i = idx / (d * Nq), r = (idx / Nq) % d, g = idx % Nq;
    double s = 0.0;
    for (int k = 0; k < m; ++k) {
      const double* o = jv + (size_t)(i * m + k) * jvs;
      if (use_x) s = fma(o[(size_t)r * Nq + g], w.xv[k * Nq + g], s);
      for (int l = 0; l < d; ++l) s = fma(o[(size_t)(d + l * d + r) * Nq + g], w.xq[(k * d + l) * Nq + g], s);
    }
    w.tv[(i * d + r) * Nq + g] = s;
  }
  for (int idx = tid; idx < m * Nfp; idx += RF_THREADS) {
    int i = idx / Nfp, fp = idx % Nfp;
    double s = 0.0;
    if (use_x) {
      if (PJ.Su)        // Roe-type: sum_k wf S_ik x_k
        for (int k = 0; k < m; ++k) s = fma(PJ.Su[((size_t)(e * m + i) * m + k) * Nfp + fp], w.xf[k * Nfp + fp], s);
      else
        s = PJ.lamw[e * Nfp + fp] * w.xf[i * Nfp + fp];
    }
    for (int k = 0; k < m; ++k) {
      const double* o = jf + (size_t)(i * m + k) * jfs;
      if (use_z) s = fma(o[fp], w.zf[k * Nfp + fp], s);
      for (int l = 0; l < d; ++l) s = fma(o[(size_t)(1 + l) * Nfp + fp], w.xqf[(k * d + l) * Nfp + fp], s);
    }
    w.tf[i * Nfp + fp] = s;
    // domain-boundary face: the trace rows see the linearised boundary flux instead
    if (tt.fkind && tt.fkind[e * dm.nf + fp / Nfq] != kFaceInterior) {
      const int nc = 2 + d;
      double tb = 0.0;
      for (int k = 0; k < m; ++k) {
        const double* jb = PJ.Jb + ((size_t)(e * m + i) * m + k) * nc * Nfp + fp;
        if (use_z) tb = fma(jb[0], w.zf[k * Nfp + fp], tb);
        if (use_x) tb = fma(jb[(size_t)Nfp], w.xf[k * Nfp + fp], tb);
        for (int l = 0; l < d; ++l) tb = fma(jb[(size_t)(2 + l) * Nfp], w.xqf[(k * d + l) * Nfp + fp], tb);
      }
      w.tbf[i * Nfp + fp] = tb;
    }
  }
  __syncthreads();
  // projections onto the test functions
  const double* Ms = G.Mass + (size_t)e * Np * Np;
  if (d == 3) {
    // sum_{g,r} Dxi_r[g][a] tv_r(g) with Dxi_0 = L'(x)L(x)L, Dxi_1 = L(x)L'(x)L, Dxi_2 = L(x)L(x)L':
    // contract z (L or L'), then y, then x
    const int np1 = dm.np1, nq1 = dm.nq1;
    const int TS = nq1 * nq1 * np1, VS = nq1 * np1 * np1;
    double* t1 = w.xq;                      // m 3 TS <= m d Nq (xq is free here)
    double* t2 = w.dqn;                     // m 2 VS <= m d Np + m Nq: dqn | xv, both free here
    // face terms sum_fp PhiF[fp][a] tf(fp) per face: first over the points' first
    // tangential index (into xqf, free now), then the second (into xf), so that
    // fb[i][f][tn] holds face f's term for its tn-th node
    const int nf = dm.nf, FB = nq1 * np1, Nfn1 = np1 * np1;
    double* fu = w.xqf;                     // m nf FB <= m d Nfp
    double* fb = w.xf;                      // m nf Nfn <= m Nfp
    for (int idx = tid; idx < m * nf * FB; idx += RF_THREADS) {
      int i = idx / (nf * FB), f = (idx / FB) % nf, t = idx % FB;
      int a0 = t % np1, g1 = t / np1;
      const double* src = w.tf + i * Nfp + f * Nfq + nq1 * g1;
      double s = 0.0;
      for (int g0 = 0; g0 < nq1; ++g0) s = fma(w.sL[g0 * np1 + a0], src[g0], s);
      fu[idx] = s;
    }
    // The mass term alpha M x = alpha Phi^T (wdet x(g)) (M formed with the same points
    // and weights) rides on direction 2: after the z stage its L (x) L part joins T_2,
    // which the y and x stages contract with L (x) L, so it costs one z stage.
    const bool mass_q = ph.alpha != 0.0 && use_x;
    const double* wd = G.wdet + (size_t)e * Nq;
    for (int idx = tid; idx < m * 3 * TS; idx += RF_THREADS) {
      int i = idx / (3 * TS), r = (idx / TS) % 3, t = idx % TS;
      int gxy = t % (nq1 * nq1), az = t / (nq1 * nq1);
      const double* X = r == 2 ? w.sdL : w.sL;
      const double* src = w.tv + (i * d + r) * Nq + gxy;
      double s = 0.0;
      for (int gz = 0; gz < nq1; ++gz) s = fma(X[gz * np1 + az], src[nq1 * nq1 * gz], s);
      if (r == 2 && mass_q) {
        const double* xg = w.xv + i * Nq + gxy;
        double sm2 = 0.0;
        for (int gz = 0; gz < nq1; ++gz)
          sm2 = fma(w.sL[gz * np1 + az], wd[gxy + nq1 * nq1 * gz] * xg[nq1 * nq1 * gz], sm2);
        s = fma(ph.alpha, sm2, s);
      }
      t1[idx] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < m * VS; idx += RF_THREADS) {
      int i = idx / VS, t = idx % VS;
      int gx = t % nq1, ay = (t / nq1) % np1, az = t / (nq1 * np1);
      const double* T0 = t1 + (i * 3 + 0) * TS;
      const double* T1 = t1 + (i * 3 + 1) * TS;
      const double* T2 = t1 + (i * 3 + 2) * TS;
      double s0 = 0.0, s1 = 0.0;
      for (int gy = 0; gy < nq1; ++gy) {
        int tt = gx + nq1 * (gy + nq1 * az);
        double Ly = w.sL[gy * np1 + ay], dLy = w.sdL[gy * np1 + ay];
        s0 = fma(Ly, T0[tt], s0);
        s1 = fma(dLy, T1[tt], s1);
        s1 = fma(Ly, T2[tt], s1);
      }
      t2[(i * 2 + 0) * VS + t] = s0;
      t2[(i * 2 + 1) * VS + t] = s1;
    }
    for (int idx = tid; idx < m * nf * Nfn1; idx += RF_THREADS) {
      int i = idx / (nf * Nfn1), f = (idx / Nfn1) % nf, tn = idx % Nfn1;
      int a0 = tn % np1, a1 = tn / np1;
      const double* src = fu + ((size_t)i * nf + f) * FB + a0;
      double s = 0.0;
      for (int g1 = 0; g1 < nq1; ++g1) s = fma(w.sL[g1 * np1 + a1], src[np1 * g1], s);
      fb[idx] = s;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < m * Np; idx += RF_THREADS) {
    int i = idx / Np, a = idx % Np;
    double s = 0.0;
    if (d != 3 && ph.alpha != 0.0 && use_x) {     // 3D: in the projection stages above
      double t = 0.0;
      for (int b = 0; b < Np; ++b) t = fma(Ms[a * Np + b], w.x[i * Np + b], t);
      s = ph.alpha * t;
    }
    if (d == 3) {
      const int np1 = dm.np1, nq1 = dm.nq1, VS = nq1 * np1 * np1;
      int ax = a % np1, ay = (a / np1) % np1, az = a / (np1 * np1);
      const double* V0 = w.dqn + (i * 2 + 0) * VS;
      const double* V1 = w.dqn + (i * 2 + 1) * VS;
      for (int gx = 0; gx < nq1; ++gx) {
        int t = gx + nq1 * (ay + np1 * az);
        s = fma(w.sdL[gx * np1 + ax], V0[t], s);
        s = fma(w.sL[gx * np1 + ax], V1[t], s);
      }
    } else {
      for (int g = 0; g < Nq; ++g)
        for (int r = 0; r < d; ++r)
          s = fma(ref.Dxi[((size_t)r * Nq + g) * Np + a], w.tv[(i * d + r) * Nq + g], s);
    }
    if (ref.slot[a] >= 0) {
      if (d == 3) {
        s += face_part(dm, w.xf, i, a);
      } else {
        for (int fp = 0; fp < Nfp; ++fp) s = fma(ref.PhiF[(size_t)fp * Np + a], w.tf[i * Nfp + fp], s);
      }
    }
    w.ou[idx] = s;
  }
  for (int idx = tid; idx < m * Nb; idx += RF_THREADS) {
    int i = idx / Nb, sl = idx % Nb;
    double s = 0.0;
    if (tt.sfl) {
      if (sl < nbe) {
        const int* fl = tt.sfl + ((size_t)e * Nb + sl) * 3;
        for (int c = 0; c < 3; ++c) {
          const int code = fl[c];
          if (code < 0) continue;
          const int f = code / tt.NFS, j = code % tt.NFS;
          const double* mu = tt.muf + ((size_t)e * dm.nf + f) * Nfq * tt.NFS + j;
          const double* src = (tt.fkind && tt.fkind[e * dm.nf + f] != kFaceInterior) ? w.tbf : w.tf;
          for (int gf = 0; gf < Nfq; ++gf) s = fma(mu[(size_t)gf * tt.NFS], src[i * Nfp + f * Nfq + gf], s);
        }
      }
    } else if (d == 3) {
      // uniform order, every face interior (meshes with boundary faces carry the slot
      // tables above): the trace basis on a face is the element basis there, so the
      // trace row of slot sl is the face part of the u-row of its node
      s = face_part(dm, w.xf, i, ref.bnode[sl]);
    } else {
      const int a = ref.bnode[sl];
      for (int fp = 0; fp < Nfp; ++fp) s = fma(ref.PhiF[(size_t)fp * Np + a], w.tf[i * Nfp + fp], s);
    }
    w.ot[idx] = s;
  }
  __syncthreads();
}

// f <- (I_m (x) L^-1) f (transpose = false) or (I_m (x) L^-T) f, L^-1 lower triangular
// [Np][Np]; tmp holds nu floats.
__device__ void mass_apply(const Dims& dm, const float* __restrict__ Linv, float* f, float* tmp, bool transpose) {
  const int Np = dm.Np;
  for (int r = threadIdx.x; r < dm.nu; r += RF_THREADS) {
    const int i = r / Np, a = r % Np;
    const float* fi = f + i * Np;
    float s = 0.f;
    if (!transpose)
      for (int b = 0; b <= a; ++b) s = fmaf(Linv[a * Np + b], fi[b], s);
    else
      for (int b = a; b < Np; ++b) s = fmaf(Linv[b * Np + a], fi[b], s);
    tmp[r] = s;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < dm.nu; r += RF_THREADS) f[r] = tmp[r];
  __syncthreads();
}

// Asynchronous 16-byte global -> shared copies (L2 only), completion per thread.
__device__ __forceinline__ void cp_async16(float* sdst, const float* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(sdst))),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Row r, columns kb .. kb + 31, of the FP32 factors into the thread's slot (16-byte
// pieces: ld, kb and the element offsets are multiples of 4 floats; kb + 32 <= ld).
__device__ __forceinline__ void stage_row(const float* __restrict__ A, int ld, int r, int kb, float* slot) {
  const float* src = A + (int64_t)r * ld + kb;
#pragma unroll
  for (int c = 0; c < RF_NB / 4; ++c) cp_async16(slot + 4 * c, src + 4 * c);
}

// v <- A~32^-1 v with the FP32 factors in the form k_solve_prep leaves them: each
// 32 x 32 diagonal block holds [L11^-1 \ U11^-1] and pp the panels' interchanges
// composed into gathers.  A correction only needs FP32 accuracy (the residual it
// corrects is FP64), so the solve runs in FP32 on a scaled copy of v held in f (nu
// floats, any free shared buffer with nu more floats behind it).  Per panel of the
// forward solve: the interchanges as one gather, x = L11^-1 (gathered values) by warp 0
// from its row of the inverted block, then rows below -= L21 x; the backward solve
// runs the panels in reverse with x = U11^-1 f and rows above -= U12 x.  Warp 0 uses
// its row of the diagonal block and every other thread the 32 factor entries of the row
// it updates, staged in its shared-memory slot (stg, 16-byte aligned) by asynchronous
// copies issued one panel ahead, as soon as the slot's previous row has been used, so
// that their latency overlaps the panel steps.  Rows past the first of a thread (nu >
// RF_THREADS - 32) are read directly.
// With a mass scaling (Linv != null) the factors are those of S A~ S^T, S = I (x) L^-1,
// and A~^-1 = S^T (S A~ S^T)^-1 S; f + nu serves as the scratch of the two products.
__device__ void solve32(const Dims& dm, const float* __restrict__ A, int ld, const int* __restrict__ pp, double* v,
                        float* f, float* stg, double* red, const float* __restrict__ Linv) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nu = dm.nu;
  constexpr int NR = RF_THREADS - 32;            // threads that update rows (warps 1 ..)
  float* slot = stg + tid * RF_SLOT;
  const float4* slot4 = reinterpret_cast<const float4*>(slot);
  // the row a thread uses in the forward panel kb (-1: none)
  auto fwd_row = [&](int kb) {
    const int nb = min(RF_NB, nu - kb);
    if (warp == 0) return lane < nb ? kb + lane : -1;
    const int r = kb + nb + (tid - 32);
    return r < nu ? r : -1;
  };
  auto bwd_row = [&](int kb) {
    const int nb = min(RF_NB, nu - kb);
    if (warp == 0) return lane < nb ? kb + lane : -1;
    return tid - 32 < kb ? tid - 32 : -1;
  };
  {
    const int r = fwd_row(0);
    if (r >= 0) stage_row(A, ld, r, 0, slot);
  }
  double mx = 0.0;
  for (int i = tid; i < nu; i += RF_THREADS) mx = fmax(mx, fabs(v[i]));
  mx = block_max(mx, red);
  const double sc = mx > 0.0 ? mx : 1.0;
  for (int i = tid; i < nu; i += RF_THREADS) f[i] = (float)(v[i] / sc);
  __syncthreads();
  if (Linv) mass_apply(dm, Linv, f, f + nu, false);
  const int last = ((nu - 1) / RF_NB) * RF_NB;
  // this lane's part of a forward panel's gather record (warps 0 and 1), read one panel ahead
  int g_src = 0, g_dst = -1, g_osrc = 0;
  auto load_rec = [&](int kb) {
    const int nb = min(RF_NB, nu - kb);
    const int* rec = pp + 3 * kb;
    if (warp == 0 && lane < nb) g_src = rec[lane];
    g_dst = -1;
    if (warp == 1 && lane < nb) { g_dst = rec[nb + lane]; g_osrc = rec[2 * nb + lane]; }
  };
  load_rec(0);
  for (int kb = 0; kb < nu; kb += RF_NB) {
    const int nb = min(RF_NB, nu - kb);
    // the next row of this thread's slot: the next forward panel, else the first backward one
    const int kn = kb + RF_NB < nu ? kb + RF_NB : last;
    const int rn = kb + RF_NB < nu ? fwd_row(kn) : bwd_row(kn);
    // the interchanges: old values first
    float a = 0.f, ob = 0.f;
    const int dst = g_dst;
    if (warp == 0 && lane < nb) a = f[g_src];
    if (dst >= 0) ob = f[g_osrc];
    if (warp < 2 && kb + RF_NB < nu) load_rec(kb + RF_NB);
    __syncthreads();
    if (warp == 0) {
      // x_lane = a_lane + sum_{i < lane} (L11^-1)[lane][i] a_i
      cp_async_wait_all();
      float x = a;
#pragma unroll
      for (int c = 0; c < RF_NB / 4; ++c) {
        const float4 q = lane < nb ? slot4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int i = 4 * c + t;
          const float ai = __shfl_sync(0xffffffffu, a, i);
          if (i < lane) x = fmaf(qv[t], ai, x);
        }
      }
      if (rn >= 0) stage_row(A, ld, rn, kn, slot);
      if (lane < nb) f[kb + lane] = x;
    }
    if (warp == 1 && dst >= 0) f[dst] = ob;
    __syncthreads();
    if (warp > 0) {
      // full panel here (nb = 32): only the last panel can be narrower, and no row lies below it
      const int r0 = kb + nb + (tid - 32);
      if (r0 < nu) {
        cp_async_wait_all();
        float s = f[r0];
#pragma unroll
        for (int c = 0; c < RF_NB / 4; ++c) {
          const float4 q = slot4[c];
          s = fmaf(-q.x, f[kb + 4 * c + 0], s);
          s = fmaf(-q.y, f[kb + 4 * c + 1], s);
          s = fmaf(-q.z, f[kb + 4 * c + 2], s);
          s = fmaf(-q.w, f[kb + 4 * c + 3], s);
        }
        f[r0] = s;
      }
      if (rn >= 0) stage_row(A, ld, rn, kn, slot);
      for (int r = r0 + NR; r < nu; r += NR) {
        const float4* row4 = reinterpret_cast<const float4*>(A + (int64_t)r * ld + kb);
        float s = f[r];
#pragma unroll
        for (int c = 0; c < RF_NB / 4; ++c) {
          const float4 q = row4[c];
          s = fmaf(-q.x, f[kb + 4 * c + 0], s);
          s = fmaf(-q.y, f[kb + 4 * c + 1], s);
          s = fmaf(-q.z, f[kb + 4 * c + 2], s);
          s = fmaf(-q.w, f[kb + 4 * c + 3], s);
        }
        f[r] = s;
      }
    }
    __syncthreads();
  }
  for (int kb = last; kb >= 0; kb -= RF_NB) {
    const int nb = min(RF_NB, nu - kb);
    const int kn = kb - RF_NB;
    const int rn = kn >= 0 ? bwd_row(kn) : -1;
    if (warp == 0) {
      // x_lane = sum_{lane <= i < nb} (U11^-1)[lane][i] f_i
      const float a = lane < nb ? f[kb + lane] : 0.f;
      cp_async_wait_all();
      float x = 0.f;
#pragma unroll
      for (int c = 0; c < RF_NB / 4; ++c) {
        const float4 q = lane < nb ? slot4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int i = 4 * c + t;
          const float ai = __shfl_sync(0xffffffffu, a, i);
          if (i >= lane && i < nb) x = fmaf(qv[t], ai, x);
        }
      }
      if (rn >= 0) stage_row(A, ld, rn, kn, slot);
      if (lane < nb) f[kb + lane] = x;
    }
    __syncthreads();
    if (warp > 0) {
      const int r0 = tid - 32;
      if (r0 < kb) {
        cp_async_wait_all();
        float s = f[r0];
        // a ragged last panel: the entries past nb are trace columns, not U12
#pragma unroll
        for (int c = 0; c < RF_NB / 4; ++c) {
          const float4 q = slot4[c];
          const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (4 * c + t < nb) s = fmaf(-qv[t], f[kb + 4 * c + t], s);
        }
        f[r0] = s;
      }
      if (rn >= 0) stage_row(A, ld, rn, kn, slot);
      for (int r = r0 + NR; r < kb; r += NR) {
        const float4* row4 = reinterpret_cast<const float4*>(A + (int64_t)r * ld + kb);
        float s = f[r];
#pragma unroll
        for (int c = 0; c < RF_NB / 4; ++c) {
          const float4 q = row4[c];
          const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (4 * c + t < nb) s = fmaf(-qv[t], f[kb + 4 * c + t], s);
        }
        f[r] = s;
      }
    }
    __syncthreads();
  }
  cp_async_wait_all();     // nothing left in flight into the work arrays (none is issued past the last panel)
  if (Linv) mass_apply(dm, Linv, f, f + nu, true);
  for (int i = tid; i < nu; i += RF_THREADS) v[i] = sc * (double)f[i];
  __syncthreads();
}

// Solve A~ x = b (b in w.b) to FP64 accuracy; on return w.x = x and w.ou, w.ot hold
// A~ x, C~ x for that x (w.z must be zero).  Returns the final relative residual.
__device__ double refine_solve(const Dims& dm, const Phys& ph, const RefTables& ref, const Geo& G,
                               const PointJac& PJ, const TraceTab& tt, int64_t e, const float* A, int ld,
                               const int* pp, Work& w, int max_iter, const float* Linv) {
  const int tid = threadIdx.x, nu = dm.nu;
  double bn = 0.0;
  for (int i = tid; i < nu; i += RF_THREADS) { w.v[i] = w.b[i]; bn = fmax(bn, fabs(w.b[i])); }
  bn = block_max(bn, w.red);
  solve32(dm, A, ld, pp, w.v, reinterpret_cast<float*>(w.ou), stage_ptr(w), w.red, Linv);
  for (int i = tid; i < nu; i += RF_THREADS) w.x[i] = w.v[i];
  __syncthreads();
  double rel = 0.0;
  for (int it = 0; it <= max_iter; ++it) {
    element_apply(dm, ph, ref, G, PJ, tt, e, w, true, false);
    double rn = 0.0;
    for (int i = tid; i < nu; i += RF_THREADS) {
      double r = w.b[i] - w.ou[i];
      w.v[i] = r;
      rn = fmax(rn, fabs(r));
    }
    rn = block_max(rn, w.red);
    rel = bn > 0.0 ? rn / bn : rn;
    if (!(rel > kRefineTol) || it == max_iter) break;   // also stops on NaN
    solve32(dm, A, ld, pp, w.v, reinterpret_cast<float*>(w.ou), stage_ptr(w), w.red, Linv);
    for (int i = tid; i < nu; i += RF_THREADS) w.x[i] += w.v[i];
    __syncthreads();
  }
  return rel;
}

constexpr int SP_WARPS = 4;        // 2 x 4 x 4.2 KB of blocks: within the static shared-memory limit

// Once per factorisation, per element, one warp per 32-wide panel of the FP32 factors
// of A~ (the solve form solve32 reads):
//  - the diagonal block [L11 \ U11] becomes [L11^-1 \ U11^-1] in place: the inverse of
//    a unit lower triangular matrix is unit lower triangular and that of an upper
//    triangular one upper triangular, so both fit the block.  Lane c forms column c of
//    each inverse by substitution (L11 y = e_c, U11 y = e_c);
//  - the panel's row interchanges (row kb + j with row p_j >= kb + j, in order of j)
//    are composed into one gather.  At offset 3 kb of the element's record: src[j]
//    (j < nb), the row whose value ends in row kb + j; then dst[j] and osrc[j], the rows
//    below the panel that receive a value and where it comes from (dst = -1 past the
//    last such row).  A pivot outside [kb + j, nu) (an element whose factorisation did
//    not run) counts as no interchange: its status already says so.
__global__ void __launch_bounds__(SP_WARPS * 32)
k_solve_prep(Dims dm, TraceTab tt, float* __restrict__ S32, const int* __restrict__ piv, int* __restrict__ pperm) {
  __shared__ float blk[SP_WARPS][RF_NB][RF_NB + 1];
  __shared__ float inv[SP_WARPS][RF_NB][RF_NB + 1];
  __shared__ int cur[SP_WARPS][RF_NB], op[SP_WARPS][RF_NB], ov[SP_WARPS][RF_NB];
  const int64_t e = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nu = dm.nu;
  float* A = S32 + (tt.soff ? tt.soff[e] : e * (int64_t)dm.n * dm.ld);
  const int ld = tt.ldv ? tt.ldv[e] : dm.ld;
  const int* pv = piv + e * (int64_t)nu;
  int* rec0 = pperm + e * 3 * (int64_t)nu;
  float (*B)[RF_NB + 1] = blk[warp];
  float (*Y)[RF_NB + 1] = inv[warp];
  for (int kb = warp * RF_NB; kb < nu; kb += SP_WARPS * RF_NB) {
    const int nb = min(RF_NB, nu - kb);
    for (int i = 0; i < nb; ++i) B[i][lane] = lane < nb ? A[(int64_t)(kb + i) * ld + kb + lane] : 0.f;
    __syncwarp();
    if (lane < nb) {
      const int c = lane;
      // L11^-1, column c below the diagonal: y_i = -(L[i][c] + sum_{c < t < i} L[i][t] y_t)
      for (int i = c + 1; i < nb; ++i) {
        float sacc = B[i][c];
        for (int t = c + 1; t < i; ++t) sacc = fmaf(B[i][t], Y[t][c], sacc);
        Y[i][c] = -sacc;
      }
      // U11^-1, column c on and above the diagonal: y_c = 1 / U[c][c],
      // y_i = -(sum_{i < t <= c} U[i][t] y_t) / U[i][i]
      Y[c][c] = 1.f / B[c][c];
      for (int i = c - 1; i >= 0; --i) {
        float sacc = 0.f;
        for (int t = i + 1; t <= c; ++t) sacc = fmaf(B[i][t], Y[t][c], sacc);
        Y[i][c] = -sacc / B[i][i];
      }
    }
    if (lane == 0) {
      int nout = 0;
      for (int j = 0; j < nb; ++j) cur[warp][j] = kb + j;
      for (int j = 0; j < nb; ++j) {
        const int p = pv[kb + j];
        if (p <= kb + j || p >= nu) continue;
        int* slot;
        if (p < kb + nb) {
          slot = &cur[warp][p - kb];
        } else {
          int qi = 0;
          while (qi < nout && op[warp][qi] != p) ++qi;
          if (qi == nout) { op[warp][qi] = p; ov[warp][qi] = p; ++nout; }
          slot = &ov[warp][qi];
        }
        const int t = cur[warp][j];
        cur[warp][j] = *slot;
        *slot = t;
      }
      for (int j = nout; j < nb; ++j) op[warp][j] = -1;
    }
    __syncwarp();
    for (int i = 0; i < nb; ++i)
      if (lane < nb) A[(int64_t)(kb + i) * ld + kb + lane] = Y[i][lane];
    int* rec = rec0 + 3 * kb;
    if (lane < nb) {
      rec[lane] = cur[warp][lane];
      rec[nb + lane] = op[warp][lane];
      rec[2 * nb + lane] = op[warp][lane] >= 0 ? ov[warp][lane] : 0;
    }
    __syncwarp();
  }
}

// One CTA per element: y = A~^-1 F~ refined, R_e = G~ - C~ y.
__global__ void __launch_bounds__(RF_THREADS, 2)
k_refine(Dims dm, Phys ph, RefTables ref, Geo G, PointJac PJ, TraceTab tt, const float* __restrict__ S32,
         const int* __restrict__ pperm, const double* __restrict__ rhs64, double* __restrict__ y64,
         double* __restrict__ re64, int8_t* __restrict__ status, int max_iter, const float* __restrict__ Linv32) {
  extern __shared__ double sm[];
  Work w = carve(dm, sm);
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  for (int i = tid; i < dm.nq1 * dm.np1; i += RF_THREADS) { w.sL[i] = ref.L1[i]; w.sdL[i] = ref.dL1[i]; }
  const double* rhs = rhs64 + e * dm.n;
  for (int i = tid; i < dm.nu; i += RF_THREADS) w.b[i] = rhs[i];
  for (int i = tid; i < dm.nt; i += RF_THREADS) w.z[i] = 0.0;
  __syncthreads();
  const float* A = S32 + (tt.soff ? tt.soff[e] : e * (int64_t)dm.n * dm.ld);
  const int ld = tt.ldv ? tt.ldv[e] : dm.ld;
  double rel = refine_solve(dm, ph, ref, G, PJ, tt, e, A, ld, pperm + e * 3 * dm.nu, w, max_iter,
                            Linv32 ? Linv32 + e * (int64_t)dm.Np * dm.Np : nullptr);
  for (int i = tid; i < dm.nu; i += RF_THREADS) y64[e * dm.nu + i] = w.x[i];
  // trace rows of the right-hand side: packed by the element's slot count
  const int nbe = tt.nb ? tt.nb[e] : dm.Nb;
  for (int i = tid; i < dm.nt; i += RF_THREADS) {
    const int c = i / dm.Nb, sl = i % dm.Nb;
    re64[e * dm.nt + i] = sl < nbe ? rhs[dm.nu + c * nbe + sl] - w.ot[i] : 0.0;
  }
  if (tid == 0 && !(rel <= kRefineFlag) && status[e] == IEDG_ELEM_OK) status[e] = IEDG_ELEM_REFINE;
}

// One CTA per element: du = A~^-1 (F~ - B~ dU_e) refined, dq = (q* - q) - G_l du + H_l dU_e.
__global__ void __launch_bounds__(RF_THREADS, 2)
k_backsub_mixed(Dims dm, Phys ph, RefTables ref, Geo G, PointJac PJ, TraceTab tt, const int64_t* __restrict__ etrace,
                const float* __restrict__ S32, const int* __restrict__ pperm, const double* __restrict__ rhs64,
                const double* __restrict__ rhoq, const double* __restrict__ duhat, double* __restrict__ du,
                double* __restrict__ dq, int max_iter, const float* __restrict__ Linv32) {
  extern __shared__ double sm[];
  Work w = carve(dm, sm);
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  const int m = dm.m, d = dm.d, Np = dm.Np, Nb = dm.Nb;
  const int nbe = tt.nb ? tt.nb[e] : Nb;
  for (int i = tid; i < dm.nq1 * dm.np1; i += RF_THREADS) { w.sL[i] = ref.L1[i]; w.sdL[i] = ref.dL1[i]; }
  for (int i = tid; i < dm.nu; i += RF_THREADS) w.x[i] = 0.0;
  for (int i = tid; i < dm.nt; i += RF_THREADS) {
    int k = i / Nb, t = i % Nb;
    w.z[i] = t < nbe ? duhat[etrace[e * Nb + t] * m + k] : 0.0;
  }
  __syncthreads();
  element_apply(dm, ph, ref, G, PJ, tt, e, w, false, true);  // ou = B~ dU_e
  const double* rhs = rhs64 + e * dm.n;
  for (int i = tid; i < dm.nu; i += RF_THREADS) w.b[i] = rhs[i] - w.ou[i];
  for (int i = tid; i < dm.nt; i += RF_THREADS) w.z[i] = 0.0;   // solve with z = 0
  __syncthreads();
  const float* A = S32 + (tt.soff ? tt.soff[e] : e * (int64_t)dm.n * dm.ld);
  const int ld = tt.ldv ? tt.ldv[e] : dm.ld;
  refine_solve(dm, ph, ref, G, PJ, tt, e, A, ld, pperm + e * 3 * dm.nu, w, max_iter,
               Linv32 ? Linv32 + e * (int64_t)dm.Np * dm.Np : nullptr);
  for (int i = tid; i < dm.nt; i += RF_THREADS) {          // dU_e again, for dq
    int k = i / Nb, t = i % Nb;
    w.z[i] = t < nbe ? duhat[etrace[e * Nb + t] * m + k] : 0.0;
  }
  __syncthreads();
  for (int idx = tid; idx < Np * m; idx += RF_THREADS) {
    int b = idx / m, k = idx % m;
    du[e * Np * m + idx] = w.x[k * Np + b];
  }
  for (int idx = tid; idx < Np * m * d; idx += RF_THREADS) {
    int c = idx / (m * d), k = (idx / d) % m, l = idx % d;
    const double* gl = G.Gl + (((size_t)e * d + l) * Np + c) * Np;
    const double* hl = G.Hl + (((size_t)e * d + l) * Np + c) * Nb;
    double s = -rhoq[e * Np * m * d + idx];
    for (int b = 0; b < Np; ++b) s = fma(-gl[b], w.x[k * Np + b], s);
    for (int t = 0; t < nbe; ++t) s = fma(hl[t], w.z[k * Nb + t], s);
    dq[e * Np * m * d + idx] = s;
  }
}

}  // namespace

cudaError_t launch_solve_prep(iedg_mesh* M, cudaStream_t st) {
  const Dims& dm = M->dm;
  // solve32 reads 32 columns from every panel start, the last one included
  if (((dm.nu - 1) / RF_NB) * RF_NB + RF_NB > dm.n + 1 || !M->pperm) return cudaErrorInvalidValue;
  k_solve_prep<<<(unsigned)M->E, SP_WARPS * 32, 0, st>>>(dm, M->tt, M->S32, M->piv, M->pperm);
  return cudaGetLastError();
}

cudaError_t launch_refine(iedg_mesh* M, cudaStream_t st) {
  const Dims& dm = M->dm;
  size_t smem = sizeof(double) * work_doubles(dm);
  cudaError_t err = cudaFuncSetAttribute(k_refine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_refine<<<(unsigned)M->E, RF_THREADS, smem, st>>>(dm, M->ph, M->ref, M->geo, M->pj, M->tt, M->S32, M->pperm, M->rhs64,
                                                      M->y64, M->re64, M->status, refine_iters(M),
                                                      M->mass_scaled ? M->Linv32 : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_backsub_mixed(iedg_mesh* M, const double* duhat, double* du, double* dq, cudaStream_t st) {
  const Dims& dm = M->dm;
  size_t smem = sizeof(double) * work_doubles(dm);
  cudaError_t err = cudaFuncSetAttribute(k_backsub_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_backsub_mixed<<<(unsigned)M->E, RF_THREADS, smem, st>>>(dm, M->ph, M->ref, M->geo, M->pj, M->tt, M->etrace, M->S32,
                                                             M->pperm, M->rhs64, M->rhoq, duhat, du, dq,
                                                             refine_iters(M), M->mass_scaled ? M->Linv32 : nullptr);
  return cudaGetLastError();
}

}  // namespace iedg
