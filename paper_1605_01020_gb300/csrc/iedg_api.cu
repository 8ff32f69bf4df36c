// C ABI of the IEDG library: handle creation (reference element, geometry,
// trace-matrix pattern, gather lists, workspace) and the compute entry points.
// The sequence of kernels behind each entry point is described in iedg.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "iedg_internal.cuh"

using namespace iedg;

static std::string g_err;   // failures before a handle exists

// ------------------------------------------------------------------------------
// Reference element (host).  Gauss-Legendre points are the roots of P_n found by
// Newton's method; Gauss-Lobatto-Legendre nodes are +-1 and the roots of P_p'
// (Newton's method with the Legendre differential equation for P_p'').  The basis
// is the tensor product of 1D Lagrange polynomials through the GLL nodes.
// ------------------------------------------------------------------------------
namespace {

void legendre_eval(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1; p1 = p2;
  }
  *P = p1;
  *dP = n * (p0 - x * p1) / (1.0 - x * x);
}

void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n); w.resize(n);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_eval(n, t, &P, &dP);
      double dt = P / dP;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double P, dP;
    legendre_eval(n, t, &P, &dP);
    x[n - 1 - i] = t;                       // ascending order
    w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
}

void lobatto_nodes(int p, std::vector<double>& x) {
  x.assign(p + 1, 0.0);
  x[0] = -1.0; x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double t = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_eval(p, t, &P, &dP);
      double d2 = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
      double dt = dP / d2;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
}

// l_j(x) and l_j'(x) for the Lagrange polynomials through `nodes`.
void lagrange_eval(const std::vector<double>& nodes, double x, double* L, double* dL) {
  int n = (int)nodes.size();
  for (int j = 0; j < n; ++j) {
    double v = 1.0, dv = 0.0;
    for (int k = 0; k < n; ++k) {
      if (k == j) continue;
      double f = 1.0 / (nodes[j] - nodes[k]);
      dv = dv * (x - nodes[k]) * f + v * f;   // product rule, accumulated left to right
      v *= (x - nodes[k]) * f;
    }
    L[j] = v; dL[j] = dv;
  }
}

struct HostRef {
  std::vector<double> Phi, Dxi, Wq, PhiF, DxiF, Wf, L1, dL1;
  std::vector<int> bnode, slot, fnode;
};

HostRef build_reference(const Dims& dm) {
  HostRef R;
  const int d = dm.d, np1 = dm.np1, nq1 = dm.nq1;
  std::vector<double> xn, xq, wq;
  lobatto_nodes(dm.p, xn);
  gauss_rule(nq1, xq, wq);
  std::vector<double> L(nq1 * np1), dL(nq1 * np1);
  for (int g = 0; g < nq1; ++g) lagrange_eval(xn, xq[g], &L[g * np1], &dL[g * np1]);
  R.L1 = L;
  R.dL1 = dL;
  auto idx = [&](int a, int r, int n1) { for (int t = 0; t < r; ++t) a /= n1; return a % n1; };
  R.Phi.assign((size_t)dm.Nq * dm.Np, 1.0);
  R.Dxi.assign((size_t)d * dm.Nq * dm.Np, 1.0);
  R.Wq.assign(dm.Nq, 1.0);
  for (int g = 0; g < dm.Nq; ++g) {
    for (int r = 0; r < d; ++r) R.Wq[g] *= wq[idx(g, r, nq1)];
    for (int a = 0; a < dm.Np; ++a)
      for (int r = 0; r < d; ++r) {
        int gi = idx(g, r, nq1), ai = idx(a, r, np1);
        R.Phi[(size_t)g * dm.Np + a] *= L[gi * np1 + ai];
        for (int s = 0; s < d; ++s)
          R.Dxi[((size_t)s * dm.Nq + g) * dm.Np + a] *= (s == r ? dL : L)[gi * np1 + ai];
      }
  }
  // faces: the face-normal factor is exactly 0 or 1 at xi_r = -1 (node 0) / +1 (node p);
  // its derivative is the 1D Lagrange derivative at the end point.
  std::vector<double> Le(2 * np1), dLe(2 * np1);
  lagrange_eval(xn, -1.0, &Le[0], &dLe[0]);
  lagrange_eval(xn, 1.0, &Le[np1], &dLe[np1]);
  for (int j = 0; j < np1; ++j) { Le[j] = (j == 0); Le[np1 + j] = (j == dm.p); }
  R.Wf.assign(dm.Nfq, 1.0);
  for (int gf = 0; gf < dm.Nfq; ++gf)
    for (int t = 0; t < d - 1; ++t) R.Wf[gf] *= wq[idx(gf, t, nq1)];
  R.PhiF.assign((size_t)dm.Nfp * dm.Np, 1.0);
  R.DxiF.assign((size_t)d * dm.Nfp * dm.Np, 1.0);
  for (int f = 0; f < dm.nf; ++f) {
    int r = f / 2, side = f % 2;
    for (int gf = 0; gf < dm.Nfq; ++gf) {
      int fp = f * dm.Nfq + gf;
      for (int a = 0; a < dm.Np; ++a) {
        int t = 0;
        for (int s = 0; s < d; ++s) {
          int ai = idx(a, s, np1);
          double v, dv;
          if (s == r) { v = Le[side * np1 + ai]; dv = dLe[side * np1 + ai]; }
          else { int gi = idx(gf, t++, nq1); v = L[gi * np1 + ai]; dv = dL[gi * np1 + ai]; }
          R.PhiF[(size_t)fp * dm.Np + a] *= v;
          for (int s2 = 0; s2 < d; ++s2)
            R.DxiF[((size_t)s2 * dm.Nfp + fp) * dm.Np + a] *= (s2 == s ? dv : v);
        }
      }
    }
  }
  R.slot.assign(dm.Np, -1);
  for (int a = 0; a < dm.Np; ++a) {
    bool b = false;
    for (int r = 0; r < d; ++r) { int ai = idx(a, r, np1); b = b || ai == 0 || ai == dm.p; }
    if (b) { R.slot[a] = (int)R.bnode.size(); R.bnode.push_back(a); }
  }
  for (int f = 0; f < dm.nf; ++f) {
    int r = f / 2, side = f % 2;
    for (int a = 0; a < dm.Np; ++a)
      if (idx(a, r, np1) == (side ? dm.p : 0)) R.fnode.push_back(a);
  }
  return R;
}

Dims make_dims(int d, int p, int quad_extra) {
  Dims dm{};
  dm.d = d; dm.p = p; dm.m = d + 2; dm.np1 = p + 1; dm.nq1 = p + quad_extra;
  dm.Np = 1; dm.Nq = 1; dm.Nfq = 1; dm.Nfn = 1;
  int inner = 1;
  for (int r = 0; r < d; ++r) { dm.Np *= dm.np1; dm.Nq *= dm.nq1; inner *= (p - 1); }
  for (int r = 0; r < d - 1; ++r) { dm.Nfq *= dm.nq1; dm.Nfn *= dm.np1; }
  dm.Nb = dm.Np - inner;
  dm.nf = 2 * d;
  dm.Nfp = dm.nf * dm.Nfq;
  dm.nu = dm.m * dm.Np;
  dm.nt = dm.m * dm.Nb;
  dm.n = dm.nu + dm.nt;
  dm.ld = (dm.n + 1 + 3) & ~3;        // rows start on 16-byte boundaries (float4 / double2 access)
  return dm;
}

int fail(iedg_mesh* M, int code, const std::string& msg) {
  if (M) M->err = msg; else g_err = msg;
  return code;
}

template <class T>
cudaError_t dalloc(iedg_mesh* M, T** p, size_t count) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e == cudaSuccess) { M->allocs.push_back(*p); M->ws_bytes += (int64_t)bytes; }
  return e;
}

template <class T>
cudaError_t upload(iedg_mesh* M, T** p, const std::vector<T>& h, cudaStream_t st) {
  cudaError_t e = dalloc(M, p, h.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

void free_all(iedg_mesh* M) {
  for (void* p : M->allocs) cudaFree(p);
  M->allocs.clear();
}

}  // namespace

#define CUDA_TRY(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      int code_ = (e_ == cudaErrorMemoryAllocation) ? IEDG_ERR_OOM : IEDG_ERR_CUDA; \
      return fail(M, code_, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    }                                                                               \
  } while (0)

// Counts the launch of kernel `name`; while profiling, brackets it with events
// recorded on the launching stream.
template <class F>
static cudaError_t traced(iedg_mesh* M, const char* name, cudaStream_t st, F&& launch) {
  int id = -1;
  for (size_t i = 0; i < M->kname.size(); ++i)
    if (M->kname[i] == name) { id = (int)i; break; }
  if (id < 0) {
    id = (int)M->kname.size();
    M->kname.emplace_back(name);
    M->klaunch.push_back(0);
    M->kms.push_back(0.0);
  }
  M->klaunch[id]++;
  if (!M->profiling) return launch();
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&b);
  if (e != cudaSuccess) { cudaEventDestroy(a); return e; }
  cudaEventRecord(a, st);
  e = launch();
  cudaEventRecord(b, st);
  M->kev.push_back({id, {a, b}});
  return e;
}
#define TRACED(name, call) traced(M, name, st, [&]() { return (call); })

static void drain_events(iedg_mesh* M) {
  for (auto& pe : M->kev) {
    float ms = 0.f;
    if (cudaEventSynchronize(pe.second.second) == cudaSuccess &&
        cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess)
      M->kms[pe.first] += ms;
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  M->kev.clear();
}

// ------------------------------------------------------------------------------
extern "C" const char* iedg_last_error(const iedg_mesh* mesh) {
  return mesh ? mesh->err.c_str() : g_err.c_str();
}

static int create_impl(const iedg_mesh_desc* D, cudaStream_t st, iedg_mesh* M) {
  const Dims& dm = M->dm;
  const int64_t E = M->E, T = M->T;
  // element -> trace map checks
  const int64_t* et = D->elem_trace;
  for (int64_t i = 0; i < E * dm.Nb; ++i)
    if (et[i] < 0 || et[i] >= T) return fail(M, IEDG_ERR_MESH, "elem_trace entry out of range");
  // trace pattern: node -> elements, then union of element trace sets per node
  std::vector<int64_t> ne_ptr(T + 1, 0);
  for (int64_t i = 0; i < E * dm.Nb; ++i) ne_ptr[et[i] + 1]++;
  for (int64_t t = 0; t < T; ++t) ne_ptr[t + 1] += ne_ptr[t];
  {
    std::vector<char> seen(T, 0);
    for (int64_t t = 0; t < T; ++t)
      if (ne_ptr[t + 1] == ne_ptr[t]) return fail(M, IEDG_ERR_MESH, "trace node used by no element");
    (void)seen;
  }
  std::vector<int64_t> rc_src(E * dm.Nb);
  {
    std::vector<int64_t> fill(ne_ptr.begin(), ne_ptr.end() - 1);
    for (int64_t e = 0; e < E; ++e)       // element order => deterministic sums
      for (int s = 0; s < dm.Nb; ++s) rc_src[fill[et[e * dm.Nb + s]]++] = e * dm.Nb + s;
  }
  std::vector<int64_t> row_ptr(T + 1, 0);
  std::vector<int32_t> col;
  {
    std::vector<int64_t> mark(T, -1);
    std::vector<int32_t> buf;
    for (int64_t r = 0; r < T; ++r) {
      buf.clear();
      for (int64_t k = ne_ptr[r]; k < ne_ptr[r + 1]; ++k) {
        int64_t e = rc_src[k] / dm.Nb;
        for (int s = 0; s < dm.Nb; ++s) {
          int64_t c = et[e * dm.Nb + s];
          if (mark[c] != r) { mark[c] = r; buf.push_back((int32_t)c); }
        }
      }
      std::sort(buf.begin(), buf.end());
      col.insert(col.end(), buf.begin(), buf.end());
      row_ptr[r + 1] = (int64_t)col.size();
    }
  }
  M->nnzb = (int64_t)col.size();
  // K gather lists, stable in element order
  std::vector<int64_t> kc_ptr(M->nnzb + 1, 0);
  std::vector<int64_t> kc_blk((size_t)E * dm.Nb * dm.Nb);
  for (int64_t e = 0; e < E; ++e)
    for (int s = 0; s < dm.Nb; ++s) {
      int64_t r = et[e * dm.Nb + s];
      const int32_t* cb = col.data() + row_ptr[r];
      int64_t len = row_ptr[r + 1] - row_ptr[r];
      for (int t = 0; t < dm.Nb; ++t) {
        int32_t c = (int32_t)et[e * dm.Nb + t];
        int64_t k = row_ptr[r] + (std::lower_bound(cb, cb + len, c) - cb);
        kc_blk[(e * dm.Nb + s) * dm.Nb + t] = k;
        kc_ptr[k + 1]++;
      }
    }
  for (int64_t k = 0; k < M->nnzb; ++k) kc_ptr[k + 1] += kc_ptr[k];
  std::vector<int64_t> kc_src(kc_blk.size());
  {
    std::vector<int64_t> fill(kc_ptr.begin(), kc_ptr.end() - 1);
    for (int64_t i = 0; i < (int64_t)kc_blk.size(); ++i) kc_src[fill[kc_blk[i]]++] = i;
  }
  std::vector<int64_t>().swap(kc_blk);
  std::vector<int64_t> etv(et, et + E * dm.Nb);

  HostRef R = build_reference(dm);
  CUDA_TRY(upload(M, &M->ref.Phi, R.Phi, st));
  CUDA_TRY(upload(M, &M->ref.Dxi, R.Dxi, st));
  CUDA_TRY(upload(M, &M->ref.Wq, R.Wq, st));
  CUDA_TRY(upload(M, &M->ref.PhiF, R.PhiF, st));
  CUDA_TRY(upload(M, &M->ref.DxiF, R.DxiF, st));
  CUDA_TRY(upload(M, &M->ref.Wf, R.Wf, st));
  CUDA_TRY(upload(M, &M->ref.bnode, R.bnode, st));
  CUDA_TRY(upload(M, &M->ref.slot, R.slot, st));
  CUDA_TRY(upload(M, &M->ref.fnode, R.fnode, st));
  CUDA_TRY(upload(M, &M->ref.L1, R.L1, st));
  CUDA_TRY(upload(M, &M->ref.dL1, R.dL1, st));
  CUDA_TRY(upload(M, &M->etrace, etv, st));
  CUDA_TRY(upload(M, &M->row_ptr, row_ptr, st));
  CUDA_TRY(upload(M, &M->col, col, st));
  CUDA_TRY(upload(M, &M->kc_ptr, kc_ptr, st));
  CUDA_TRY(upload(M, &M->kc_src, kc_src, st));
  std::vector<int64_t> rc_ptr(ne_ptr);
  CUDA_TRY(upload(M, &M->rc_ptr, rc_ptr, st));
  CUDA_TRY(upload(M, &M->rc_src, rc_src, st));

  const size_t d = dm.d, Np = dm.Np, Nq = dm.Nq, Nb = dm.Nb, Nfp = dm.Nfp, m = dm.m;
  Geo& G = M->geo;
  CUDA_TRY(dalloc(M, &G.wdet, E * Nq));
  CUDA_TRY(dalloc(M, &G.Jinv, E * Nq * d * d));
  CUDA_TRY(dalloc(M, &G.fw, E * Nfp));
  CUDA_TRY(dalloc(M, &G.fn, E * Nfp * d));
  CUDA_TRY(dalloc(M, &G.Mass, E * Np * Np));
  CUDA_TRY(dalloc(M, &G.Gl, E * d * Np * Np));
  CUDA_TRY(dalloc(M, &G.Hl, E * d * Np * Nb));
  CUDA_TRY(dalloc(M, &G.GlV, E * d * Nq * Np));
  CUDA_TRY(dalloc(M, &G.HlV, E * d * Nq * Nb));
  CUDA_TRY(dalloc(M, &G.GlF, E * d * Nfp * Np));
  CUDA_TRY(dalloc(M, &G.HlF, E * d * Nfp * Nb));
  CUDA_TRY(dalloc(M, &M->pj.Jv, E * m * m * (1 + d) * d * Nq));
  CUDA_TRY(dalloc(M, &M->pj.Jf, E * m * m * (1 + d) * Nfp));
  CUDA_TRY(dalloc(M, &M->pj.lamw, E * Nfp));
  CUDA_TRY(dalloc(M, &M->qstar, E * Np * m * d));
  CUDA_TRY(dalloc(M, &M->rhoq, E * Np * m * d));
  CUDA_TRY(dalloc(M, &M->rhat, E * Nb * m));
  if (M->precision == IEDG_PRECISION_FP64) {
    CUDA_TRY(dalloc(M, &M->S, (size_t)E * dm.n * dm.ld));
  } else {
    CUDA_TRY(dalloc(M, &M->S32, (size_t)E * dm.n * dm.ld));
    CUDA_TRY(dalloc(M, &M->piv, (size_t)E * dm.nu));
    CUDA_TRY(dalloc(M, &M->rhs64, (size_t)E * dm.n));
    CUDA_TRY(dalloc(M, &M->y64, (size_t)E * dm.nu));
    CUDA_TRY(dalloc(M, &M->re64, (size_t)E * dm.nt));
    CUDA_TRY(dalloc(M, &M->pj.Jv32, E * m * m * (1 + d) * d * Nq));
    CUDA_TRY(dalloc(M, &M->pj.Jf32, E * m * m * (1 + d) * Nfp));
    CUDA_TRY(dalloc(M, &M->pj.lamw32, E * Nfp));
    CUDA_TRY(dalloc(M, &G.Mass32, E * Np * Np));
    CUDA_TRY(dalloc(M, &G.GlV32, E * d * Nq * Np));
    CUDA_TRY(dalloc(M, &G.HlV32, E * d * Nq * Nb));
    CUDA_TRY(dalloc(M, &G.GlF32, E * d * Nfp * Np));
    CUDA_TRY(dalloc(M, &G.HlF32, E * d * Nfp * Nb));
    CUDA_TRY(dalloc(M, &M->ref.Phi32, Nq * Np));
    CUDA_TRY(dalloc(M, &M->ref.Dxi32, d * Nq * Np));
    CUDA_TRY(dalloc(M, &M->ref.PhiF32, Nfp * Np));
  }
  CUDA_TRY(dalloc(M, &M->status, E));
  CUDA_TRY(dalloc(M, &M->dev_flag, 1));
  CUDA_TRY(dalloc(M, &M->queue, 1));
  CUDA_TRY(dalloc(M, &M->kry, (size_t)(IEDG_MAX_RESTART + 3) * T * m));
  CUDA_TRY(dalloc(M, &M->dinv, (size_t)T * m * m));
  CUDA_TRY(dalloc(M, &M->kpart, (size_t)(IEDG_MAX_RESTART + 1) * 512));
  CUDA_TRY(dalloc(M, &M->khdev, (size_t)(IEDG_MAX_RESTART + 1)));
  CUDA_TRY(cudaMemsetAsync(M->dev_flag, 0, sizeof(int), st));
  CUDA_TRY(cudaMemsetAsync(M->status, 0, E, st));

  // geometry: node coordinates and a scratch for B_l, E_l, freed afterwards
  double* X = nullptr;
  double* scratch = nullptr;
  CUDA_TRY(cudaMalloc(&X, E * Np * d * sizeof(double)));
  cudaError_t e1 = cudaMalloc(&scratch, E * d * Np * (Np + Nb) * sizeof(double));
  if (e1 != cudaSuccess) { cudaFree(X); CUDA_TRY(e1); }
  cudaError_t e2 = cudaMemcpyAsync(X, D->node_xyz, E * Np * d * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e2 == cudaSuccess) e2 = launch_geometry(M, X, scratch, st);
  if (e2 == cudaSuccess && M->precision == IEDG_PRECISION_MIXED) {
    const std::pair<const double*, float*> cv[] = {
        {G.Mass, G.Mass32}, {G.GlV, G.GlV32}, {G.HlV, G.HlV32}, {G.GlF, G.GlF32}, {G.HlF, G.HlF32},
        {M->ref.Phi, M->ref.Phi32}, {M->ref.Dxi, M->ref.Dxi32}, {M->ref.PhiF, M->ref.PhiF32}};
    const int64_t E_ = E, Np_ = (int64_t)Np, Nq_ = (int64_t)Nq, Nb_ = (int64_t)Nb, Nfp_ = (int64_t)Nfp,
                  d_ = (int64_t)d;
    const int64_t cn[] = {E_ * Np_ * Np_, E_ * d_ * Nq_ * Np_, E_ * d_ * Nq_ * Nb_, E_ * d_ * Nfp_ * Np_,
                          E_ * d_ * Nfp_ * Nb_, Nq_ * Np_, d_ * Nq_ * Np_, Nfp_ * Np_};
    for (int i = 0; i < 8 && e2 == cudaSuccess; ++i) e2 = launch_to_f32(cv[i].first, cv[i].second, cn[i], st);
  }
  int flag = 0;
  if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(&flag, M->dev_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
  cudaFree(X);
  cudaFree(scratch);
  CUDA_TRY(e2);
  if (flag) return fail(M, IEDG_ERR_MESH, "element with detJ <= 0 at a quadrature point");
  return IEDG_OK;
}

extern "C" int iedg_create_mesh(const iedg_mesh_desc* D, void* stream, iedg_mesh** out) {
  iedg_mesh* M = nullptr;
  if (!D || !out) return fail(M, IEDG_ERR_INVALID_ARG, "null descriptor or output");
  *out = nullptr;
  if (!(D->dim == 2 || D->dim == 3)) return fail(M, IEDG_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (D->order < 1 || D->order > (D->dim == 3 ? 4 : 3))
    return fail(M, IEDG_ERR_UNSUPPORTED, "order must be 1..4 (3D) or 1..3 (2D)");
  if (D->quad_extra < 1 || D->quad_extra > 3)
    return fail(M, IEDG_ERR_UNSUPPORTED, "quad_extra must be 1..3");
  if (D->precision != IEDG_PRECISION_FP64 && D->precision != IEDG_PRECISION_MIXED)
    return fail(M, IEDG_ERR_UNSUPPORTED, "precision must be IEDG_PRECISION_FP64 or IEDG_PRECISION_MIXED");
  if (D->stab != 0) return fail(M, IEDG_ERR_UNSUPPORTED, "only Lax-Friedrichs stabilisation is built");
  if (D->n_elem <= 0 || D->n_trace <= 0 || !D->node_xyz || !D->elem_trace)
    return fail(M, IEDG_ERR_INVALID_ARG, "empty mesh or null mesh arrays");
  if (!(D->gamma > 1.0) || !(D->Pr > 0) || !(D->Re > 0) || !(D->alpha >= 0))
    return fail(M, IEDG_ERR_INVALID_ARG, "physical parameters out of range");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return fail(M, IEDG_ERR_CUDA, "no CUDA device");
  M = new iedg_mesh();
  M->dm = make_dims(D->dim, D->order, D->quad_extra);
  M->ph = Phys{D->gamma, D->Pr, D->Re, D->alpha};
  M->precision = D->precision;
  M->E = D->n_elem;
  M->T = D->n_trace;
  int rc = create_impl(D, (cudaStream_t)stream, M);
  if (rc != IEDG_OK) {
    g_err = M->err;
    free_all(M);
    delete M;
    return rc;
  }
  *out = M;
  return IEDG_OK;
}

extern "C" int iedg_destroy_mesh(iedg_mesh* M) {
  if (!M) return IEDG_ERR_INVALID_ARG;
  drain_events(M);
  free_all(M);
  delete M;
  return IEDG_OK;
}

extern "C" int iedg_mesh_info(const iedg_mesh* M, int32_t* Np, int32_t* Nb, int64_t* nnzb,
                              int64_t* ws) {
  if (!M) return IEDG_ERR_INVALID_ARG;
  if (Np) *Np = M->dm.Np;
  if (Nb) *Nb = M->dm.Nb;
  if (nnzb) *nnzb = M->nnzb;
  if (ws) *ws = M->ws_bytes;
  return IEDG_OK;
}

extern "C" int iedg_trace_pattern(const iedg_mesh* Mc, int64_t* row_ptr, int32_t* col, void* stream) {
  iedg_mesh* M = const_cast<iedg_mesh*>(Mc);
  if (!M || !row_ptr || !col) return fail(M, IEDG_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(row_ptr, M->row_ptr, (M->T + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(col, M->col, M->nnzb * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  return IEDG_OK;
}

extern "C" int iedg_eval_residual(iedg_mesh* M, const double* u, const double* uhat, const double* q,
                                  const double* u_ref, double* q_out, double* r_q, double* r_u,
                                  double* r_fl, void* stream) {
  if (!M || !u || !uhat) return fail(M, IEDG_ERR_INVALID_ARG, "null argument");
  if (!q && !q_out) return fail(M, IEDG_ERR_INVALID_ARG, "q_out required when q is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const Dims& dm = M->dm;
  const double* qq = q;
  if (!q) {
    CUDA_TRY(TRACED("lift", launch_lift(M, u, uhat, q_out, st)));
    qq = q_out;
  } else if (q_out) {
    CUDA_TRY(cudaMemcpyAsync(q_out, q, M->E * dm.Np * dm.m * dm.d * sizeof(double),
                             cudaMemcpyDeviceToDevice, st));
  }
  if (r_q) {
    if (q) CUDA_TRY(TRACED("lift", launch_lift(M, u, uhat, M->qstar, st)));
    CUDA_TRY(TRACED("rq", launch_rq(M, qq, q ? M->qstar : qq, r_q, nullptr, st)));
  }
  if (r_u || r_fl) {
    CUDA_TRY(TRACED("points_residual", launch_points(M, u, qq, nullptr, uhat, u_ref, false, r_u, M->rhat, st)));
    if (r_fl)
      CUDA_TRY(TRACED("scatter_R", launch_scatter_R(M, M->rhat, (int64_t)dm.Nb * dm.m, dm.m, 1, r_fl, st)));
  }
  return IEDG_OK;
}

extern "C" int iedg_assemble_condensed(iedg_mesh* M, const double* u, const double* q,
                                       const double* uhat, const double* u_ref, double* K,
                                       double* R, void* stream) {
  if (!M || !u || !q || !uhat || !K || !R) return fail(M, IEDG_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const Dims& dm = M->dm;
  CUDA_TRY(cudaMemsetAsync(M->status, 0, M->E, st));
  CUDA_TRY(TRACED("lift", launch_lift(M, u, uhat, M->qstar, st)));
  CUDA_TRY(TRACED("rq", launch_rq(M, q, M->qstar, nullptr, M->rhoq, st)));
  // point Jacobians at (u, q) and the right-hand sides F~ = -R_u(u, q*), G~ = -R_FL,e(u, q*)
  // written straight into the last column of the bordered element matrices
  CUDA_TRY(TRACED("points_jacobian", launch_points(M, u, q, M->qstar, uhat, u_ref, true, nullptr, nullptr, st)));
  if (assemble_sf_supported(dm))
    CUDA_TRY(TRACED("assemble", launch_assemble_sf(M, st)));
  else
    CUDA_TRY(TRACED("assemble", launch_assemble(M, st)));
  CUDA_TRY(TRACED("lu_schur", launch_lu(M, st)));
  if (M->precision == IEDG_PRECISION_MIXED) CUDA_TRY(TRACED("refine", launch_refine(M, st)));
  CUDA_TRY(TRACED("scatter_K", launch_scatter_K(M, K, st)));
  if (M->precision == IEDG_PRECISION_FP64)
    CUDA_TRY(TRACED("scatter_R", launch_scatter_R(M, M->S + (int64_t)dm.nu * dm.ld + dm.n, (int64_t)dm.n * dm.ld,
                                                  dm.ld, (int64_t)dm.Nb * dm.ld, R, st)));
  else
    CUDA_TRY(TRACED("scatter_R", launch_scatter_R(M, M->re64, dm.nt, 1, dm.Nb, R, st)));
  M->assembled = true;
  return IEDG_OK;
}

extern "C" int iedg_back_substitute(iedg_mesh* M, const double* duhat, double* du, double* dq,
                                    void* stream) {
  if (!M || !duhat || !du || !dq) return fail(M, IEDG_ERR_INVALID_ARG, "null argument");
  if (!M->assembled) return fail(M, IEDG_ERR_NOT_ASSEMBLED, "back-substitution before assembly");
  cudaStream_t st = (cudaStream_t)stream;
  if (M->precision == IEDG_PRECISION_FP64)
    CUDA_TRY(TRACED("backsub", launch_backsub(M, duhat, du, dq, st)));
  else
    CUDA_TRY(TRACED("backsub", launch_backsub_mixed(M, duhat, du, dq, st)));
  return IEDG_OK;
}

extern "C" int64_t iedg_element_status(iedg_mesh* M, int8_t* out, void* stream) {
  if (!M || !out) return fail(M, IEDG_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(out, M->status, M->E, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  int64_t n = 0;
  for (int64_t e = 0; e < M->E; ++e) n += out[e] != 0;
  return n;
}

extern "C" int iedg_profile_enable(iedg_mesh* M, int32_t enable) {
  if (!M) return IEDG_ERR_INVALID_ARG;
  M->profiling = enable != 0;
  return IEDG_OK;
}

extern "C" int iedg_profile_read(iedg_mesh* M, int32_t max_kernels, char* names, int64_t* launches,
                                 double* ms, int32_t* n_kernels) {
  if (!M || max_kernels < 0 || (max_kernels > 0 && (!names || !launches || !ms)))
    return fail(M, IEDG_ERR_INVALID_ARG, "bad profile_read arguments");
  drain_events(M);
  int32_t n = (int32_t)M->kname.size();
  for (int32_t i = 0; i < n && i < max_kernels; ++i) {
    std::memset(names + 32 * i, 0, 32);
    std::strncpy(names + 32 * i, M->kname[i].c_str(), 31);
    launches[i] = M->klaunch[i];
    ms[i] = M->kms[i];
  }
  if (n_kernels) *n_kernels = n;
  return IEDG_OK;
}

extern "C" int iedg_profile_reset(iedg_mesh* M) {
  if (!M) return IEDG_ERR_INVALID_ARG;
  drain_events(M);
  for (auto& c : M->klaunch) c = 0;
  for (auto& t : M->kms) t = 0.0;
  return IEDG_OK;
}

extern "C" int iedg_get_schedule(const iedg_mesh* M, iedg_schedule* out) {
  if (!M || !out) return IEDG_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->lu_persistent = M->sched.lu_persistent;
  out->lu_panel = M->sched.lu_panel;
  out->asm_chunk = M->sched.asm_chunk;
  return IEDG_OK;
}

extern "C" int iedg_set_schedule(iedg_mesh* M, const iedg_schedule* in) {
  if (!M || !in) return fail(M, IEDG_ERR_INVALID_ARG, "null argument");
  if ((in->lu_persistent != 0 && in->lu_persistent != 1) || (in->lu_panel != 16 && in->lu_panel != 32) ||
      (in->asm_chunk != 0 && in->asm_chunk != 8 && in->asm_chunk != 16 && in->asm_chunk != 32))
    return fail(M, IEDG_ERR_INVALID_ARG, "schedule values out of range");
  M->sched.lu_persistent = in->lu_persistent;
  M->sched.lu_panel = in->lu_panel;
  M->sched.asm_chunk = in->asm_chunk;
  return IEDG_OK;
}
