// Quadrature-point physics and residual of the IEDG weak form.
//
//  * Navier-Stokes flux F(u, q) (Sec. 2.1): inviscid part rho v_j, rho v_i v_j +
//    delta_ij p, v_j (rho E + p); viscous part tau_ij = (1/Re)(d_j v_i + d_i v_j -
//    2/3 delta_ij d_k v_k); heat term (gamma / (Re Pr)) d_j e with e = E - |v|^2/2,
//    taken with the dissipative sign (the energy flux loses v_i tau_ij + it).
//  * Lax-Friedrichs numerical flux (Eq. IEDG d): fhat = F(uhat, q) n + lambda (u -
//    uhat), lambda = |vhat . n| + chat evaluated at uhat.
//  * Pointwise Jacobians by forward-mode dual numbers, m directions per pass:
//    one pass over u (or uhat), one pass per gradient direction l over q_{., l}.
//  * Residual projections (Eq. IEDG b, c):
//      R_u[a][i]  = sum_{g,r} Dxi_r[g][a] fvol[i][r][g] + sum_g Phi[g][a] mvol[i][g]
//                 + sum_fp PhiF[fp][a] fsur[i][fp]
//      Rhat[s][i] = sum_fp PhiF[fp][bnode[s]] fsur[i][fp]
//    with fvol = -w Jinv[r][j] F_ij, mvol = alpha w (u - u_ref)_i, fsur = wf fhat_i.
//  * R_q = M (q - q*) where q* = H_l uhat - G_l u is the lifted gradient that makes
//    R_q vanish (Eq. IEDG a is linear: R_q = M q + B_l u - E_l uhat).
#include <type_traits>

#include "iedg_internal.cuh"

namespace iedg {
namespace {

// ------------------------------------------------------------------ dual numbers
template <int N>
struct Dual {
  double v;
  double t[N];
};

template <int N>
__device__ inline Dual<N> mkconst(double v) {
  Dual<N> r;
  r.v = v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.t[k] = 0.0;
  return r;
}
template <int N>
__device__ inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.t[k] = a.t[k] + b.t[k];
  return r;
}
template <int N>
__device__ inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.t[k] = a.t[k] - b.t[k];
  return r;
}
template <int N>
__device__ inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.t[k] = a.t[k] * b.v + a.v * b.t[k];
  return r;
}
template <int N>
__device__ inline Dual<N> operator*(double a, const Dual<N>& b) {
  Dual<N> r; r.v = a * b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.t[k] = a * b.t[k];
  return r;
}
template <int N>
__device__ inline Dual<N> operator+(const Dual<N>& a, double b) {
  Dual<N> r = a; r.v += b; return r;
}
template <int N>
__device__ inline Dual<N> recip(const Dual<N>& a) {
  Dual<N> r; r.v = 1.0 / a.v;
  double s = -r.v * r.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.t[k] = s * a.t[k];
  return r;
}
template <int N>
__device__ inline Dual<N> dsqrt(const Dual<N>& a) {
  Dual<N> r; r.v = sqrt(a.v);
  double s = 0.5 / r.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.t[k] = s * a.t[k];
  return r;
}
template <int N>
__device__ inline Dual<N> dabs(const Dual<N>& a) {
  double s = a.v > 0 ? 1.0 : (a.v < 0 ? -1.0 : 0.0);   // sign(0) := 0
  Dual<N> r; r.v = fabs(a.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.t[k] = s * a.t[k];
  return r;
}
__device__ inline double recip(double a) { return 1.0 / a; }
__device__ inline double dsqrt(double a) { return sqrt(a); }
__device__ inline double dabs(double a) { return fabs(a); }
template <class T> __device__ inline T mk(double v);
template <> __device__ inline double mk<double>(double v) { return v; }
template <> __device__ inline Dual<4> mk<Dual<4>>(double v) { return mkconst<4>(v); }
template <> __device__ inline Dual<5> mk<Dual<5>>(double v) { return mkconst<5>(v); }

// Navier-Stokes flux F[i][j], i < M = D + 2, j < D.
template <int D, class T>
__device__ void ns_flux(const T* u, const T (*q)[D], const Phys& ph, T (*F)[D]) {
  constexpr int M = D + 2;
  const T rinv = recip(u[0]);
  T v[D];
#pragma unroll
  for (int i = 0; i < D; ++i) v[i] = u[1 + i] * rinv;
  const T E = u[M - 1] * rinv;
  T vv = v[0] * v[0];
#pragma unroll
  for (int i = 1; i < D; ++i) vv = vv + v[i] * v[i];
  const T p = (ph.gamma - 1.0) * (u[M - 1] - 0.5 * (u[0] * vv));
  T dv[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) dv[i][j] = (q[1 + i][j] - v[i] * q[0][j]) * rinv;
  T div = dv[0][0];
#pragma unroll
  for (int k = 1; k < D; ++k) div = div + dv[k][k];
  const double ire = 1.0 / ph.Re, kap = ph.gamma / (ph.Re * ph.Pr);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    T de = (q[M - 1][j] - E * q[0][j]) * rinv;
#pragma unroll
    for (int k = 0; k < D; ++k) de = de - v[k] * dv[k][j];
    F[0][j] = u[1 + j];
    T fe = v[j] * (u[M - 1] + p) - kap * de;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      T tau = dv[i][j] + dv[j][i];
      if (i == j) tau = tau - (2.0 / 3.0) * div;
      tau = ire * tau;
      T fm = u[1 + i] * v[j] - tau;
      if (i == j) fm = fm + p;
      F[1 + i][j] = fm;
      fe = fe - v[i] * tau;
    }
    F[M - 1][j] = fe;
  }
}

template <int D, class T>
__device__ T lf_lambda(const T* u, const double* n, const Phys& ph) {
  constexpr int M = D + 2;
  const T rinv = recip(u[0]);
  T vn = mk<T>(0.0), vv = mk<T>(0.0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    T vj = u[1 + j] * rinv;
    vn = vn + n[j] * vj;
    vv = vv + vj * vj;
  }
  T p = (ph.gamma - 1.0) * (u[M - 1] - 0.5 * (u[0] * vv));
  return dabs(vn) + dsqrt((ph.gamma * p) * rinv);
}

// Roe-type stabilisation out = |A_n(uh)| du, A_n the normal Jacobian of the Euler flux
// at uh (Sec. 2.1).  Eigenvalues v_n - c, v_n (d-fold), v_n + c; the acoustic waves of
// du have strengths a_-+ = (dp -+ c rho dv_n) / (2 c^2), with the linearised jumps
// dp = (gamma-1)(d(rhoE) - v.d(rho v) + |v|^2/2 drho), rho dv_n = n.d(rho v) - v_n drho,
// and eigenvectors (1, v -+ c n, H -+ c v_n); all other waves move at v_n:
//   |A_n| du = |v_n| du + (|v_n - c| - |v_n|) a_- r_- + (|v_n + c| - |v_n|) a_+ r_+ .
// T = double, or Dual<M> to differentiate with respect to uh (du may depend on it).
template <int D, class T>
__device__ void roe_apply(const T* uh, const T* du, const double* n, const Phys& ph, T* out) {
  constexpr int M = D + 2;
  const T rinv = recip(uh[0]);
  T v[D];
#pragma unroll
  for (int j = 0; j < D; ++j) v[j] = uh[1 + j] * rinv;
  T vn = mk<T>(0.0), q2 = mk<T>(0.0), vdm = mk<T>(0.0), ndm = mk<T>(0.0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    vn = vn + n[j] * v[j];
    q2 = q2 + v[j] * v[j];
    vdm = vdm + v[j] * du[1 + j];
    ndm = ndm + n[j] * du[1 + j];
  }
  const T p = (ph.gamma - 1.0) * (uh[M - 1] + (-0.5) * (uh[0] * q2));
  const T c2 = ph.gamma * (p * rinv);
  const T c = dsqrt(c2);
  const T H = (uh[M - 1] + p) * rinv;
  const T dp = (ph.gamma - 1.0) * (du[M - 1] + (-1.0) * vdm + 0.5 * (q2 * du[0]));
  const T rdvn = ndm + (-1.0) * (vn * du[0]);
  const T ic2 = 0.5 * recip(c2);
  const T am = (dp + (-1.0) * (c * rdvn)) * ic2;
  const T ap = (dp + c * rdvn) * ic2;
  const T l0 = dabs(vn);
  const T wm = (dabs(vn + (-1.0) * c) + (-1.0) * l0) * am;
  const T wp = (dabs(vn + c) + (-1.0) * l0) * ap;
  out[0] = l0 * du[0] + wm + wp;
#pragma unroll
  for (int j = 0; j < D; ++j) out[1 + j] = l0 * du[1 + j] + wm * (v[j] + (-n[j]) * c) + wp * (v[j] + n[j] * c);
  out[M - 1] = l0 * du[M - 1] + wm * (H + (-1.0) * (c * vn)) + wp * (H + c * vn);
}

// out = A_n(uh) x, A_n = d(F_inv . n)/du the normal Jacobian of the Euler flux at uh,
// from the differentials of rho v_n, rho v v_n + p n, (rho E + p) v_n with
// dp = (gamma-1)(x_E - v.x_m + |v|^2/2 x_rho) and H = (rho E + p)/rho.
template <int D, class T>
__device__ void normal_jac_apply(const T* uh, const T* x, const double* n, const Phys& ph, T* out) {
  constexpr int M = D + 2;
  const T rinv = recip(uh[0]);
  T v[D];
#pragma unroll
  for (int j = 0; j < D; ++j) v[j] = uh[1 + j] * rinv;
  T vn = mk<T>(0.0), q2 = mk<T>(0.0), vdm = mk<T>(0.0), ndm = mk<T>(0.0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    vn = vn + n[j] * v[j];
    q2 = q2 + v[j] * v[j];
    vdm = vdm + v[j] * x[1 + j];
    ndm = ndm + n[j] * x[1 + j];
  }
  const T p = (ph.gamma - 1.0) * (uh[M - 1] + (-0.5) * (uh[0] * q2));
  const T H = (uh[M - 1] + p) * rinv;
  const T dp = (ph.gamma - 1.0) * (x[M - 1] + (-1.0) * vdm + 0.5 * (q2 * x[0]));
  out[0] = ndm;
#pragma unroll
  for (int j = 0; j < D; ++j) out[1 + j] = x[1 + j] * vn + v[j] * ndm + (-1.0) * (v[j] * (vn * x[0])) + n[j] * dp;
  out[M - 1] = (x[M - 1] + dp) * vn + H * (ndm + (-1.0) * (vn * x[0]));
}

// Far-field boundary flux (Sec. 2.1): bhat = (A_n + |A_n|)/2 (uh - u) + (A_n - |A_n|)/2
// (uh - u_b), A_n and |A_n| at uh.  T = double or Dual<M> (uh seeded; u, u_b constant).
template <int D, class T>
__device__ void farfield_flux(const T* uh, const double* u, const double* ub, const double* n, const Phys& ph,
                              T* b) {
  constexpr int M = D + 2;
  T a[M], c[M], Aa[M], Sa[M], Ac[M], Sc[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    a[i] = uh[i] + mk<T>(-u[i]);
    c[i] = uh[i] + mk<T>(-ub[i]);
  }
  normal_jac_apply<D, T>(uh, a, n, ph, Aa);
  roe_apply<D, T>(uh, a, n, ph, Sa);
  normal_jac_apply<D, T>(uh, c, n, ph, Ac);
  roe_apply<D, T>(uh, c, n, ph, Sc);
#pragma unroll
  for (int i = 0; i < M; ++i) b[i] = 0.5 * (Aa[i] + Sa[i]) + 0.5 * (Ac[i] + (-1.0) * Sc[i]);
}

// Boundary flux of the trace equation at one face point of kind fk (far field or
// no-slip adiabatic wall): wf bhat into bval[M] and, with jac, the point's entries of
// Jb.  A wall's energy row is the energy row of fhat, whose derivatives the calling
// thread wrote to Jf, Su / lamw just before; they are read back here.
template <int D, int STAB>
__device__ __noinline__ void boundary_point(int fk, const double* uh, const double* u, const double* n, double wf,
                                            const Phys& ph, double fhatE, bool jac, const PointJac& PJ, int64_t e,
                                            int fp, int Nfp, double* bval) {
  constexpr int M = D + 2, NC = 2 + D;
  const size_t jfs = (size_t)(1 + D) * Nfp;
  auto jb = [&](int i, int k, int c) -> size_t { return (((size_t)(e * M + i) * M + k) * NC + c) * Nfp + fp; };
  auto put = [&](int i, int k, int c, double v) {
    PJ.Jb[jb(i, k, c)] = v;
    if (PJ.Jb32) PJ.Jb32[jb(i, k, c)] = (float)v;
  };
  if (fk == kFaceFarField) {
    double b[M];
    farfield_flux<D, double>(uh, u, ph.ub, n, ph, b);
#pragma unroll
    for (int i = 0; i < M; ++i) bval[i] = wf * b[i];
    if (!jac) return;
    Dual<M> ud[M], bd[M];
#pragma unroll
    for (int k = 0; k < M; ++k) { ud[k] = mkconst<M>(uh[k]); ud[k].t[k] = 1.0; }
    farfield_flux<D, Dual<M>>(ud, u, ph.ub, n, ph, bd);
#pragma unroll 1
    for (int k = 0; k < M; ++k) {
      double ek[M], Ak[M], Sk[M];
#pragma unroll
      for (int i = 0; i < M; ++i) ek[i] = (i == k) ? 1.0 : 0.0;
      normal_jac_apply<D, double>(uh, ek, n, ph, Ak);
      roe_apply<D, double>(uh, ek, n, ph, Sk);
#pragma unroll
      for (int i = 0; i < M; ++i) {
        put(i, k, 0, wf * bd[i].t[k]);
        put(i, k, 1, -0.5 * wf * (Ak[i] + Sk[i]));
#pragma unroll
        for (int l = 0; l < D; ++l) put(i, k, 2 + l, 0.0);
      }
    }
    return;
  }
  // wall: (rhohat - rho, rho vhat, fhat_E)
  bval[0] = wf * (uh[0] - u[0]);
#pragma unroll
  for (int j = 0; j < D; ++j) bval[1 + j] = wf * uh[1 + j];
  bval[M - 1] = wf * fhatE;
  if (!jac) return;
  const double* jfE = PJ.Jf + ((size_t)e * M * M + (size_t)(M - 1) * M) * jfs;   // row E of this element
#pragma unroll 1
  for (int k = 0; k < M; ++k) {
    for (int i = 0; i < M - 1; ++i) {
      put(i, k, 0, (i == k) ? wf : 0.0);
      put(i, k, 1, (i == 0 && k == 0) ? -wf : 0.0);
      for (int l = 0; l < D; ++l) put(i, k, 2 + l, 0.0);
    }
    const double* o = jfE + (size_t)k * jfs;
    put(M - 1, k, 0, o[fp]);
    double su;
    if constexpr (STAB == 1) su = PJ.Su[((size_t)(e * M + (M - 1)) * M + k) * Nfp + fp];
    else su = (k == M - 1) ? PJ.lamw[e * Nfp + fp] : 0.0;
    put(M - 1, k, 1, su);
    for (int l = 0; l < D; ++l) put(M - 1, k, 2 + l, o[(size_t)(1 + l) * Nfp + fp]);
  }
}

// The flux Jacobians at (u, q) by forward-mode duals, handed to the caller pass by pass
// so that no full dF / dQ array is held: on_u(Fd) after the pass over u, with
// Fd[i][j].t[k] = dF_ij/du_k, then on_q(l, Fd) after the pass over q_{., l}, with
// Fd[i][j].t[k] = dF_ij/dq_kl.
template <int D, class OnU, class OnQ>
__device__ __forceinline__ void flux_jacobians(const double* u, const double (*q)[D], const Phys& ph, OnU on_u,
                                               OnQ on_q) {
  constexpr int M = D + 2;
  using TD = Dual<M>;
  TD ud[M], qd[M][D], Fd[M][D];
  // pass over u
#pragma unroll
  for (int k = 0; k < M; ++k) { ud[k] = mkconst<M>(u[k]); ud[k].t[k] = 1.0; }
#pragma unroll
  for (int k = 0; k < M; ++k)
#pragma unroll
    for (int l = 0; l < D; ++l) qd[k][l] = mkconst<M>(q[k][l]);
  ns_flux<D, TD>(ud, qd, ph, Fd);
  on_u(Fd);
  // passes over q_{., l}
#pragma unroll
  for (int k = 0; k < M; ++k) ud[k] = mkconst<M>(u[k]);
#pragma unroll 1
  for (int l = 0; l < D; ++l) {
#pragma unroll
    for (int k = 0; k < M; ++k)
#pragma unroll
      for (int ll = 0; ll < D; ++ll) {
        qd[k][ll] = mkconst<M>(q[k][ll]);
        if (ll == l) qd[k][ll].t[k] = 1.0;
      }
    ns_flux<D, TD>(ud, qd, ph, Fd);
    on_q(l, Fd);
  }
}

// ------------------------------------------------------------------ point kernel
// One CTA per element.  jac = false: residual at (u, q).  jac = true: Jacobians at
// (u, q) into PointJac, right-hand sides -R_u(u, q*), -Rhat(u, q*) into the last
// column of the bordered element matrix.
// JAC is a compile-time choice so that the residual form carries none of the Jacobian
// code's registers and local arrays (it runs at a higher occupancy).
template <int D, int STAB, bool JAC>
__global__ void k_points(Dims dm, Phys ph, RefTables ref, Geo G, PointJac PJ,
                         const int64_t* __restrict__ etrace, const double* __restrict__ U,
                         const double* __restrict__ Q, const double* __restrict__ QS,
                         const double* __restrict__ UH, const double* __restrict__ UREF,
                         double* __restrict__ RU, double* __restrict__ RHAT, double* __restrict__ RHS,
                         int64_t rhs_es, int64_t rhs_rs, TraceTab tt) {
  constexpr int M = D + 2;
  constexpr bool jac = JAC;
  extern __shared__ double sm[];
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Np = dm.Np, Nq = dm.Nq, Nb = dm.Nb, Nfp = dm.Nfp, Nfq = dm.Nfq, Nfn = dm.Nfn;
  double* su = sm;                         // [Np][M]
  double* sq = su + Np * M;                // [Np][M][D]
  double* sqs = sq + Np * M * D;           // [Np][M][D]  (q* for the right-hand side)
  double* sur = sqs + Np * M * D;          // [Np][M]
  double* suh = sur + Np * M;              // [Nb][M]
  double* fvol = suh + Nb * M;             // [M][D][Nq]
  double* mvol = fvol + M * D * Nq;        // [M][Nq]
  double* fsur = mvol + M * Nq;            // [M][Nfp]
  double* ftr = fsur + M * Nfp;            // [M][Nfp]  flux of the trace rows (bhat on boundary faces)
  const bool has_ref = UREF != nullptr && ph.alpha != 0.0;
  for (int i = tid; i < Np * M; i += nth) {
    su[i] = U[e * Np * M + i];
    sur[i] = has_ref ? UREF[e * Np * M + i] : 0.0;
  }
  for (int i = tid; i < Np * M * D; i += nth) {
    sq[i] = Q[e * Np * M * D + i];
    sqs[i] = QS ? QS[e * Np * M * D + i] : sq[i];
  }
  const int nbe = tt.nb ? tt.nb[e] : Nb;         // trace slots of this element
  for (int i = tid; i < nbe * M; i += nth) {
    int s = i / M, k = i % M;
    suh[i] = UH[etrace[e * Nb + s] * M + k];
  }
  __syncthreads();
  const size_t jvs = (size_t)(1 + D) * D * Nq;    // stride of one (i,k) pair in Jv
  const size_t jfs = (size_t)(1 + D) * Nfp;
  // ---- volume points
  for (int g = tid; g < Nq; g += nth) {
    double u[M], q[M][D], qr[M][D], du[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      u[i] = 0; du[i] = 0;
#pragma unroll
      for (int j = 0; j < D; ++j) { q[i][j] = 0; qr[i][j] = 0; }
    }
    const double* phi = ref.Phi + (size_t)g * Np;
    for (int a = 0; a < Np; ++a) {
      double ph_a = phi[a];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        u[i] += ph_a * su[a * M + i];
        du[i] += ph_a * (su[a * M + i] - sur[a * M + i]);
#pragma unroll
        for (int j = 0; j < D; ++j) {
          q[i][j] += ph_a * sq[(a * M + i) * D + j];
          qr[i][j] += ph_a * sqs[(a * M + i) * D + j];
        }
      }
    }
    const double w = G.wdet[e * Nq + g];
    double Ji[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int j = 0; j < D; ++j) Ji[r][j] = G.Jinv[((e * Nq + g) * D + r) * D + j];
    double F[M][D];
    ns_flux<D, double>(u, qr, ph, F);
#pragma unroll
    for (int i = 0; i < M; ++i) {
#pragma unroll
      for (int r = 0; r < D; ++r) {
        double s = 0;
#pragma unroll
        for (int j = 0; j < D; ++j) s += Ji[r][j] * F[i][j];
        fvol[(i * D + r) * Nq + g] = -w * s;
      }
      mvol[i * Nq + g] = has_ref ? ph.alpha * w * du[i] : 0.0;
    }
    if constexpr (JAC) {
      double* jv = PJ.Jv + (size_t)e * M * M * jvs;
      float* jv32 = PJ.Jv32 ? PJ.Jv32 + (size_t)e * M * M * jvs : nullptr;
      // entry c of pair (i, k): -w sum_j Ji[r][j] dF_ij/d(unknown), c = r for u, D + l D + r for q_l
      auto put = [&](int c0, const Dual<M> (*Fd)[D]) {
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
          for (int k = 0; k < M; ++k) {
            double* o = jv + (size_t)(i * M + k) * jvs;
#pragma unroll
            for (int r = 0; r < D; ++r) {
              double s = 0;
#pragma unroll
              for (int j = 0; j < D; ++j) s += Ji[r][j] * Fd[i][j].t[k];
              o[(size_t)(c0 + r) * Nq + g] = -w * s;
              if (jv32) jv32[(size_t)(i * M + k) * jvs + (size_t)(c0 + r) * Nq + g] = (float)(-w * s);
            }
          }
      };
      flux_jacobians<D>(u, q, ph, [&](const Dual<M> (*Fd)[D]) { put(0, Fd); },
                        [&](int l, const Dual<M> (*Fd)[D]) { put(D + l * D, Fd); });
    }
  }
  // ---- face points
  for (int fp = tid; fp < Nfp; fp += nth) {
    const int f = fp / Nfq;
    double u[M], uh[M], q[M][D], qr[M][D];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      u[i] = 0; uh[i] = 0;
#pragma unroll
      for (int j = 0; j < D; ++j) { q[i][j] = 0; qr[i][j] = 0; }
    }
    const double* phi = ref.PhiF + (size_t)fp * Np;
    for (int t = 0; t < Nfn; ++t) {
      int a = ref.fnode[f * Nfn + t];
      double ph_a = phi[a];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        u[i] += ph_a * su[a * M + i];
        if (!tt.nfs) uh[i] += ph_a * suh[ref.slot[a] * M + i];
#pragma unroll
        for (int j = 0; j < D; ++j) {
          q[i][j] += ph_a * sq[(a * M + i) * D + j];
          qr[i][j] += ph_a * sqs[(a * M + i) * D + j];
        }
      }
    }
    if (tt.nfs) {
      // trace basis of this face from the element's table
      const int cnt = tt.nfs[e * dm.nf + f];
      const int* fsf = tt.fs + ((size_t)e * dm.nf + f) * tt.NFS;
      const double* mu = tt.muf + (((size_t)e * dm.nf + f) * Nfq + (fp - f * Nfq)) * tt.NFS;
      for (int j = 0; j < cnt; ++j)
#pragma unroll
        for (int i = 0; i < M; ++i) uh[i] += mu[j] * suh[fsf[j] * M + i];
    }
    const double wf = G.fw[e * Nfp + fp];
    double n[D];
#pragma unroll
    for (int j = 0; j < D; ++j) n[j] = G.fn[(e * Nfp + fp) * D + j];
    double F[M][D];
    ns_flux<D, double>(uh, qr, ph, F);
    // stabilisation S (u - uh): lambda I (Lax-Friedrichs) or |A_n(uh)| (Roe-type)
    double sdu[M];
    double lam = 0.0;
    if constexpr (STAB == 1) {
      double dd[M];
#pragma unroll
      for (int i = 0; i < M; ++i) dd[i] = u[i] - uh[i];
      roe_apply<D, double>(uh, dd, n, ph, sdu);
    } else {
      lam = lf_lambda<D, double>(uh, n, ph);
#pragma unroll
      for (int i = 0; i < M; ++i) sdu[i] = lam * (u[i] - uh[i]);
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
      double s = sdu[i];
#pragma unroll
      for (int j = 0; j < D; ++j) s += F[i][j] * n[j];
      fsur[i * Nfp + fp] = wf * s;
    }
    if (jac) {
      Dual<M> ud[M];
#pragma unroll
      for (int k = 0; k < M; ++k) { ud[k] = mkconst<M>(uh[k]); ud[k].t[k] = 1.0; }
      // d/duhat of the stabilisation term: LF  dlambda/duhat (u - uh) - lambda I;
      // Roe  d/duhat [ |A_n(uh)| (u - uh) ] by duals (includes - |A_n|)
      Dual<M> lamd = mkconst<M>(0.0);
      Dual<M> gd[M];
      if constexpr (STAB == 1) {
        Dual<M> dd[M];
#pragma unroll
        for (int i = 0; i < M; ++i) dd[i] = mkconst<M>(u[i]) - ud[i];
        roe_apply<D, Dual<M>>(ud, dd, n, ph, gd);
        // dfhat/du = S: its columns S e_k
#pragma unroll 1
        for (int k = 0; k < M; ++k) {
          double ek[M], sk[M];
#pragma unroll
          for (int i = 0; i < M; ++i) ek[i] = (i == k) ? 1.0 : 0.0;
          roe_apply<D, double>(uh, ek, n, ph, sk);
#pragma unroll
          for (int i = 0; i < M; ++i) {
            const size_t o = ((size_t)(e * M + i) * M + k) * Nfp + fp;
            PJ.Su[o] = wf * sk[i];
            if (PJ.Su32) PJ.Su32[o] = (float)(wf * sk[i]);
          }
        }
      } else {
        lamd = lf_lambda<D, Dual<M>>(ud, n, ph);
      }
      double* jf = PJ.Jf + (size_t)e * M * M * jfs;
      float* jf32 = PJ.Jf32 ? PJ.Jf32 + (size_t)e * M * M * jfs : nullptr;
      // entry 0 of pair (i, k): the stabilisation's derivative + dfhat/du n; entry 1 + l:
      // dfhat/dq_l n
      flux_jacobians<D>(
          uh, q, ph,
          [&](const Dual<M> (*Fd)[D]) {
#pragma unroll
            for (int i = 0; i < M; ++i)
#pragma unroll
              for (int k = 0; k < M; ++k) {
                double s = STAB == 1 ? gd[i].t[k] : lamd.t[k] * (u[i] - uh[i]) - (i == k ? lam : 0.0);
#pragma unroll
                for (int j = 0; j < D; ++j) s += Fd[i][j].t[k] * n[j];
                jf[(size_t)(i * M + k) * jfs + fp] = wf * s;
                if (jf32) jf32[(size_t)(i * M + k) * jfs + fp] = (float)(wf * s);
              }
          },
          [&](int l, const Dual<M> (*Fd)[D]) {
#pragma unroll
            for (int i = 0; i < M; ++i)
#pragma unroll
              for (int k = 0; k < M; ++k) {
                double t = 0;
#pragma unroll
                for (int j = 0; j < D; ++j) t += Fd[i][j].t[k] * n[j];
                jf[(size_t)(i * M + k) * jfs + (size_t)(1 + l) * Nfp + fp] = wf * t;
                if (jf32) jf32[(size_t)(i * M + k) * jfs + (size_t)(1 + l) * Nfp + fp] = (float)(wf * t);
              }
          });
      PJ.lamw[e * Nfp + fp] = wf * lam;
      if (PJ.lamw32) PJ.lamw32[e * Nfp + fp] = (float)(wf * lam);
    }
    // trace rows: fhat on interior faces, the boundary flux on domain-boundary faces
    const int fk = tt.fkind ? tt.fkind[e * dm.nf + f] : kFaceInterior;
    if (fk != kFaceInterior) {
      double bval[M];
      boundary_point<D, STAB>(fk, uh, u, n, wf, ph, fsur[(M - 1) * Nfp + fp] / wf, jac, PJ, e, fp, Nfp, bval);
#pragma unroll
      for (int i = 0; i < M; ++i) ftr[i * Nfp + fp] = bval[i];
    } else {
#pragma unroll
      for (int i = 0; i < M; ++i) ftr[i * Nfp + fp] = fsur[i * Nfp + fp];
    }
  }
  __syncthreads();
  // ---- projections onto the test functions
  const double sgn = jac ? -1.0 : 1.0;
  // right-hand side column: uniform meshes e * rhs_es, row stride rhs_rs; meshes with
  // per-element sizes: column n_e of the element's bordered matrix
  double* rhs_e = nullptr;
  int64_t rrs = rhs_rs;
  if (jac) {
    if (tt.soff && rhs_rs != 1) {
      rhs_e = RHS + tt.soff[e] + dm.nu + (int64_t)M * nbe;
      rrs = tt.ldv[e];
    } else {
      rhs_e = RHS + e * rhs_es;
    }
  }
  for (int ai = tid; ai < Np * M; ai += nth) {
    const int a = ai / M, i = ai % M;
    double s = 0;
    for (int g = 0; g < Nq; ++g) {
      double t = ref.Phi[(size_t)g * Np + a] * mvol[i * Nq + g];
#pragma unroll
      for (int r = 0; r < D; ++r) t += ref.Dxi[((size_t)r * Nq + g) * Np + a] * fvol[(i * D + r) * Nq + g];
      s += t;
    }
    if (ref.slot[a] >= 0)
      for (int fp = 0; fp < Nfp; ++fp) s += ref.PhiF[(size_t)fp * Np + a] * fsur[i * Nfp + fp];
    if (jac) rhs_e[((int64_t)i * Np + a) * rrs] = sgn * s;
    else if (RU) RU[(e * Np + a) * M + i] = s;
  }
  for (int si = tid; si < nbe * M; si += nth) {
    const int s = si / M, i = si % M;
    double t = 0;
    if (tt.nfs) {
      const int* fl = tt.sfl + ((size_t)e * Nb + s) * 3;
      for (int c = 0; c < 3; ++c) {
        const int code = fl[c];
        if (code < 0) continue;
        const int f = code / tt.NFS, j = code % tt.NFS;
        const double* mu = tt.muf + ((size_t)e * dm.nf + f) * Nfq * tt.NFS + j;
        for (int gf = 0; gf < Nfq; ++gf) t += mu[(size_t)gf * tt.NFS] * ftr[i * Nfp + f * Nfq + gf];
      }
    } else {
      const int a = ref.bnode[s];
      for (int fp = 0; fp < Nfp; ++fp) t += ref.PhiF[(size_t)fp * Np + a] * fsur[i * Nfp + fp];
    }
    if (jac) rhs_e[((int64_t)dm.nu + (int64_t)i * nbe + s) * rrs] = sgn * t;
    else RHAT[(e * Nb + s) * M + i] = t;
  }
}

// q*[e][c][k][l] = sum_t H_l[c][t] uhat_k(t) - sum_b G_l[c][b] u_k(b)
__global__ void k_lift(Dims dm, Geo G, const int64_t* __restrict__ etrace, const double* __restrict__ U,
                       const double* __restrict__ UH, double* __restrict__ QS, TraceTab tt) {
  extern __shared__ double sm[];
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Np = dm.Np, Nb = dm.Nb, m = dm.m, d = dm.d;
  double* su = sm;            // [Np][m]
  double* suh = su + Np * m;  // [Nb][m]
  for (int i = tid; i < Np * m; i += nth) su[i] = U[e * Np * m + i];
  const int nbe = tt.nb ? tt.nb[e] : Nb;
  for (int i = tid; i < nbe * m; i += nth) suh[i] = UH[etrace[e * Nb + i / m] * m + i % m];
  __syncthreads();
  for (int idx = tid; idx < Np * m * d; idx += nth) {
    int c = idx / (m * d), k = (idx / d) % m, l = idx % d;
    const double* gl = G.Gl + (((size_t)e * d + l) * Np + c) * Np;
    const double* hl = G.Hl + (((size_t)e * d + l) * Np + c) * Nb;
    double s = 0;
    for (int t = 0; t < nbe; ++t) s += hl[t] * suh[t * m + k];
    for (int b = 0; b < Np; ++b) s -= gl[b] * su[b * m + k];
    QS[e * Np * m * d + idx] = s;
  }
}

// R_q = M (q - q*), optionally rhoq = q - q*
__global__ void k_rq(Dims dm, Geo G, const double* __restrict__ Q, const double* __restrict__ QS,
                     double* __restrict__ RQ, double* __restrict__ RHOQ) {
  extern __shared__ double sm[];
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Np = dm.Np, w = dm.m * dm.d;
  double* dq = sm;   // [Np][m d]
  for (int i = tid; i < Np * w; i += nth) {
    double v = Q[e * Np * w + i] - QS[e * Np * w + i];
    dq[i] = v;
    if (RHOQ) RHOQ[e * Np * w + i] = v;
  }
  __syncthreads();
  if (!RQ) return;
  const double* Ms = G.Mass + (size_t)e * Np * Np;
  for (int idx = tid; idx < Np * w; idx += nth) {
    int a = idx / w, c = idx % w;
    double s = 0;
    for (int b = 0; b < Np; ++b) s += Ms[a * Np + b] * dq[b * w + c];
    RQ[e * Np * w + idx] = s;
  }
}

}  // namespace

cudaError_t launch_points(iedg_mesh* M, const double* u, const double* q, const double* qs,
                          const double* uhat, const double* u_ref, bool jacobians, double* r_u,
                          double* rhat, cudaStream_t st) {
  const Dims& dm = M->dm;
  size_t smem = sizeof(double) * ((size_t)dm.Np * dm.m * (2 + 2 * dm.d) + dm.Nb * dm.m +
                                  (size_t)dm.m * dm.d * dm.Nq + dm.m * dm.Nq + 2 * dm.m * dm.Nfp);
  const int threads = 128;
  // right-hand sides: column n of the FP64 bordered matrix, or the FP64 rhs array
  // (ragged FP64 matrices: the kernel adds the element's offset and n_e to S itself)
  double* rhs = M->precision == 0 ? (M->tt.soff ? M->S : M->S + dm.n) : M->rhs64;
  int64_t es = M->precision == 0 ? (int64_t)dm.n * dm.ld : dm.n;
  int64_t rs = M->precision == 0 ? dm.ld : 1;
  auto pick = [&](auto j) {
    constexpr bool J = decltype(j)::value;
    return dm.d == 2 ? (M->ph.stab == 1 ? k_points<2, 1, J> : k_points<2, 0, J>)
                     : (M->ph.stab == 1 ? k_points<3, 1, J> : k_points<3, 0, J>);
  };
  auto kern = jacobians ? pick(std::true_type{}) : pick(std::false_type{});
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<(unsigned)M->E, threads, smem, st>>>(dm, M->ph, M->ref, M->geo, M->pj, M->etrace, u, q, qs, uhat, u_ref,
                                              r_u, rhat, rhs, es, rs, M->tt);
  return cudaGetLastError();
}

cudaError_t launch_lift(iedg_mesh* M, const double* u, const double* uhat, double* qstar, cudaStream_t st) {
  const Dims& dm = M->dm;
  size_t smem = sizeof(double) * (size_t)(dm.Np + dm.Nb) * dm.m;
  k_lift<<<(unsigned)M->E, 128, smem, st>>>(dm, M->geo, M->etrace, u, uhat, qstar, M->tt);
  return cudaGetLastError();
}

cudaError_t launch_rq(iedg_mesh* M, const double* q, const double* qs, double* r_q, double* rhoq,
                      cudaStream_t st) {
  const Dims& dm = M->dm;
  size_t smem = sizeof(double) * (size_t)dm.Np * dm.m * dm.d;
  k_rq<<<(unsigned)M->E, 128, smem, st>>>(dm, M->geo, q, qs, r_q, rhoq);
  return cudaGetLastError();
}

}  // namespace iedg
