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
  std::vector<double> Phi, Dxi, Wq, PhiF, DxiF, Wf, L1, dL1, LQ;
  std::vector<double> xq;   // 1D Gauss points
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
  R.xq = xq;
  // degree-q Gauss-Lobatto Lagrange basis at the 1D Gauss points, q = 1..4, [5][nq1][5]
  R.LQ.assign((size_t)25 * nq1, 0.0);
  for (int q = 1; q <= 4; ++q) {
    std::vector<double> xl, Lq(q + 1), dLq(q + 1);
    lobatto_nodes(q, xl);
    for (int g = 0; g < nq1; ++g) {
      lagrange_eval(xl, xq[g], Lq.data(), dLq.data());
      for (int j = 0; j <= q; ++j) R.LQ[((size_t)q * nq1 + g) * 5 + j] = Lq[j];
    }
  }
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

// Trace-matrix pattern and gather lists from per-element slot lists (element e: n_e
// trace ids at lists[e], internal id ids[e]); contributions are recorded in list
// order, so every sum runs in that element order.  Packed entries: (id P + s) for
// trace rows, (id P + s) P + t for K blocks.
static int setup_pattern(iedg_mesh* M, const std::vector<const int64_t*>& lists, const std::vector<int>& lens,
                         const std::vector<int64_t>& ids, int64_t P, cudaStream_t st) {
  const int64_t E = (int64_t)lists.size(), T = M->T;
  for (int64_t e = 0; e < E; ++e)
    for (int s = 0; s < lens[e]; ++s)
      if (lists[e][s] < 0 || lists[e][s] >= T) return fail(M, IEDG_ERR_MESH, "elem_trace entry out of range");
  // trace node -> contributions
  std::vector<int64_t> ne_ptr(T + 1, 0);
  for (int64_t e = 0; e < E; ++e)
    for (int s = 0; s < lens[e]; ++s) ne_ptr[lists[e][s] + 1]++;
  for (int64_t t = 0; t < T; ++t) ne_ptr[t + 1] += ne_ptr[t];
  for (int64_t t = 0; t < T; ++t)
    if (ne_ptr[t + 1] == ne_ptr[t]) return fail(M, IEDG_ERR_MESH, "trace node used by no element");
  std::vector<int64_t> rc_src(ne_ptr[T]), rc_el(ne_ptr[T]);
  {
    std::vector<int64_t> fill(ne_ptr.begin(), ne_ptr.end() - 1);
    for (int64_t e = 0; e < E; ++e)
      for (int s = 0; s < lens[e]; ++s) {
        int64_t k = fill[lists[e][s]]++;
        rc_src[k] = ids[e] * P + s;
        rc_el[k] = e;
      }
  }
  std::vector<int64_t> row_ptr(T + 1, 0);
  std::vector<int32_t> col;
  {
    std::vector<int64_t> mark(T, -1);
    std::vector<int32_t> buf;
    for (int64_t r = 0; r < T; ++r) {
      buf.clear();
      for (int64_t k = ne_ptr[r]; k < ne_ptr[r + 1]; ++k) {
        int64_t e = rc_el[k];
        for (int s = 0; s < lens[e]; ++s) {
          int64_t c = lists[e][s];
          if (mark[c] != r) { mark[c] = r; buf.push_back((int32_t)c); }
        }
      }
      std::sort(buf.begin(), buf.end());
      col.insert(col.end(), buf.begin(), buf.end());
      row_ptr[r + 1] = (int64_t)col.size();
    }
  }
  std::vector<int64_t>().swap(rc_el);
  M->nnzb = (int64_t)col.size();
  M->max_row_blocks = 0;
  for (int64_t r = 0; r < T; ++r) M->max_row_blocks = std::max(M->max_row_blocks, row_ptr[r + 1] - row_ptr[r]);
  // K gather lists, stable in element order
  int64_t nk = 0;
  for (int64_t e = 0; e < E; ++e) nk += (int64_t)lens[e] * lens[e];
  std::vector<int64_t> kc_ptr(M->nnzb + 1, 0);
  std::vector<int64_t> kc_blk(nk), kc_val(nk);
  {
    int64_t i = 0;
    for (int64_t e = 0; e < E; ++e)
      for (int s = 0; s < lens[e]; ++s) {
        int64_t r = lists[e][s];
        const int32_t* cb = col.data() + row_ptr[r];
        int64_t len = row_ptr[r + 1] - row_ptr[r];
        for (int t = 0; t < lens[e]; ++t, ++i) {
          int32_t c = (int32_t)lists[e][t];
          int64_t k = row_ptr[r] + (std::lower_bound(cb, cb + len, c) - cb);
          kc_blk[i] = k;
          kc_val[i] = (ids[e] * P + s) * P + t;
          kc_ptr[k + 1]++;
        }
      }
  }
  for (int64_t k = 0; k < M->nnzb; ++k) kc_ptr[k + 1] += kc_ptr[k];
  std::vector<int64_t> kc_src(nk);
  {
    std::vector<int64_t> fill(kc_ptr.begin(), kc_ptr.end() - 1);
    for (int64_t i = 0; i < nk; ++i) kc_src[fill[kc_blk[i]]++] = kc_val[i];
  }
  std::vector<int64_t>().swap(kc_blk);
  std::vector<int64_t>().swap(kc_val);
  CUDA_TRY(upload(M, &M->row_ptr, row_ptr, st));
  CUDA_TRY(upload(M, &M->col, col, st));
  CUDA_TRY(upload(M, &M->kc_ptr, kc_ptr, st));
  CUDA_TRY(upload(M, &M->kc_src, kc_src, st));
  CUDA_TRY(upload(M, &M->rc_ptr, ne_ptr, st));
  CUDA_TRY(upload(M, &M->rc_src, rc_src, st));
  // the host vectors must outlive the copies
  CUDA_TRY(cudaStreamSynchronize(st));
  return IEDG_OK;
}

// Element tables of one group of elements of equal order (the whole mesh when the
// order is uniform): reference element, geometry, point tables, lifted gradients and,
// on the mixed path, the FP64 right-hand sides and refined solutions.
static int alloc_group(iedg_mesh* M, cudaStream_t st) {
  const Dims& dm = M->dm;
  const int64_t E = M->E;
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
  CUDA_TRY(upload(M, &M->ref.LQ, R.LQ, st));
  CUDA_TRY(cudaStreamSynchronize(st));

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
  if (M->ph.stab == 1) CUDA_TRY(dalloc(M, &M->pj.Su, E * m * m * Nfp));
  if (M->has_boundary) CUDA_TRY(dalloc(M, &M->pj.Jb, E * m * m * (2 + d) * Nfp));
  CUDA_TRY(dalloc(M, &M->qstar, E * Np * m * d));
  CUDA_TRY(dalloc(M, &M->rhoq, E * Np * m * d));
  if (M->precision == IEDG_PRECISION_MIXED) {
    CUDA_TRY(dalloc(M, &M->rhs64, (size_t)E * dm.n));
    CUDA_TRY(dalloc(M, &M->y64, (size_t)E * dm.nu));
    CUDA_TRY(dalloc(M, &M->pj.Jv32, E * m * m * (1 + d) * d * Nq));
    CUDA_TRY(dalloc(M, &M->pj.Jf32, E * m * m * (1 + d) * Nfp));
    CUDA_TRY(dalloc(M, &M->pj.lamw32, E * Nfp));
    if (M->ph.stab == 1) CUDA_TRY(dalloc(M, &M->pj.Su32, E * m * m * Nfp));
    if (M->has_boundary) CUDA_TRY(dalloc(M, &M->pj.Jb32, E * m * m * (2 + d) * Nfp));
    CUDA_TRY(dalloc(M, &G.Mass32, E * Np * Np));
    CUDA_TRY(dalloc(M, &G.GlV32, E * d * Nq * Np));
    CUDA_TRY(dalloc(M, &G.HlV32, E * d * Nq * Nb));
    CUDA_TRY(dalloc(M, &G.GlF32, E * d * Nfp * Np));
    CUDA_TRY(dalloc(M, &G.HlF32, E * d * Nfp * Nb));
    CUDA_TRY(dalloc(M, &M->ref.Phi32, Nq * Np));
    CUDA_TRY(dalloc(M, &M->ref.Dxi32, d * Nq * Np));
    CUDA_TRY(dalloc(M, &M->ref.PhiF32, Nfp * Np));
    CUDA_TRY(dalloc(M, &M->ref.LQ32, (size_t)25 * dm.nq1));
  }
  CUDA_TRY(dalloc(M, &M->dev_flag, 1));
  CUDA_TRY(cudaMemsetAsync(M->dev_flag, 0, sizeof(int), st));
  return IEDG_OK;
}

// Workspace of the handle that owns the element matrices and the trace space.
static int alloc_owner(iedg_mesh* M, int64_t S_elems, int64_t piv_elems, int64_t rhat_elems, int64_t re_elems,
                       cudaStream_t st) {
  const int64_t E = M->E, T = M->T;
  const int m = M->dm.m;
  if (M->precision == IEDG_PRECISION_FP64) {
    CUDA_TRY(dalloc(M, &M->S, (size_t)S_elems));
  } else {
    CUDA_TRY(dalloc(M, &M->S32, (size_t)S_elems));
    CUDA_TRY(dalloc(M, &M->piv, (size_t)piv_elems));
    CUDA_TRY(dalloc(M, &M->pperm, (size_t)3 * piv_elems));
  }
  CUDA_TRY(dalloc(M, &M->rhat, (size_t)rhat_elems));
  CUDA_TRY(dalloc(M, &M->re64, (size_t)re_elems));
  CUDA_TRY(dalloc(M, &M->status, E));
  if (M->precision != IEDG_PRECISION_FP64 && !M->mixed_orders) {
    CUDA_TRY(dalloc(M, &M->fb_S, (size_t)kFallbackSlots * M->dm.n * M->dm.ld));
    CUDA_TRY(dalloc(M, &M->fb_list, kFallbackSlots));
    CUDA_TRY(dalloc(M, &M->fb_slot, (size_t)E));
    CUDA_TRY(dalloc(M, &M->fb_status, kFallbackSlots));
    CUDA_TRY(dalloc(M, &M->fb_count, 1));
    CUDA_TRY(cudaMemsetAsync(M->fb_count, 0, sizeof(int), st));
  }
  if (!M->dev_flag) CUDA_TRY(dalloc(M, &M->dev_flag, 1));
  CUDA_TRY(dalloc(M, &M->queue, 1));
  CUDA_TRY(dalloc(M, &M->kry, (size_t)(IEDG_MAX_RESTART + 3) * T * m));
  CUDA_TRY(dalloc(M, &M->dinv, (size_t)T * m * m));
  CUDA_TRY(dalloc(M, &M->kpart, (size_t)(IEDG_MAX_RESTART + 1) * 512));
  CUDA_TRY(dalloc(M, &M->khdev, (size_t)(IEDG_MAX_RESTART + 1)));
  CUDA_TRY(dalloc(M, &M->kst, (size_t)(2 * (IEDG_MAX_RESTART + 1) + (IEDG_MAX_RESTART + 1) * IEDG_MAX_RESTART +
                                       4 * IEDG_MAX_RESTART + 1 + 8)));
  CUDA_TRY(cudaMemsetAsync(M->dev_flag, 0, sizeof(int), st));
  CUDA_TRY(cudaMemsetAsync(M->status, 0, E, st));
  return IEDG_OK;
}

// Geometry of a group from its node coordinates (HOST [E][Np][d]) and the FP32 table
// copies of the mixed path.
static int run_geometry(iedg_mesh* M, const double* node_xyz, cudaStream_t st) {
  const Dims& dm = M->dm;
  const int64_t E = M->E;
  const size_t d = dm.d, Np = dm.Np, Nq = dm.Nq, Nb = dm.Nb, Nfp = dm.Nfp;
  Geo& G = M->geo;
  double* X = nullptr;
  double* scratch = nullptr;
  CUDA_TRY(cudaMalloc(&X, E * Np * d * sizeof(double)));
  cudaError_t e1 = cudaMalloc(&scratch, E * d * Np * (Np + Nb) * sizeof(double));
  if (e1 != cudaSuccess) { cudaFree(X); CUDA_TRY(e1); }
  cudaError_t e2 = cudaMemcpyAsync(X, node_xyz, E * Np * d * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e2 == cudaSuccess) e2 = launch_geometry(M, X, scratch, st);
  if (e2 == cudaSuccess && M->precision == IEDG_PRECISION_MIXED) {
    const std::pair<const double*, float*> cv[] = {
        {G.Mass, G.Mass32}, {G.GlV, G.GlV32}, {G.HlV, G.HlV32}, {G.GlF, G.GlF32}, {G.HlF, G.HlF32},
        {M->ref.Phi, M->ref.Phi32}, {M->ref.Dxi, M->ref.Dxi32}, {M->ref.PhiF, M->ref.PhiF32},
        {M->ref.LQ, M->ref.LQ32}};
    const int64_t E_ = E, Np_ = (int64_t)Np, Nq_ = (int64_t)Nq, Nb_ = (int64_t)Nb, Nfp_ = (int64_t)Nfp,
                  d_ = (int64_t)d;
    const int64_t cn[] = {E_ * Np_ * Np_, E_ * d_ * Nq_ * Np_, E_ * d_ * Nq_ * Nb_, E_ * d_ * Nfp_ * Np_,
                          E_ * d_ * Nfp_ * Nb_, Nq_ * Np_, d_ * Nq_ * Np_, Nfp_ * Np_, 25 * (int64_t)dm.nq1};
    for (int i = 0; i < 9 && e2 == cudaSuccess; ++i) e2 = launch_to_f32(cv[i].first, cv[i].second, cn[i], st);
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

static int create_impl(const iedg_mesh_desc* D, cudaStream_t st, iedg_mesh* M) {
  const Dims& dm = M->dm;
  const int64_t E = M->E;
  const int64_t* et = D->elem_trace;
  std::vector<const int64_t*> lists(E);
  std::vector<int> lens(E, dm.Nb);
  std::vector<int64_t> ids(E);
  for (int64_t e = 0; e < E; ++e) { lists[e] = et + e * dm.Nb; ids[e] = e; }
  M->nb_pack = dm.Nb;
  int rc = setup_pattern(M, lists, lens, ids, dm.Nb, st);
  if (rc != IEDG_OK) return rc;
  std::vector<int64_t> etv(et, et + E * dm.Nb);
  CUDA_TRY(upload(M, &M->etrace, etv, st));
  rc = alloc_group(M, st);
  if (rc != IEDG_OK) return rc;
  rc = alloc_owner(M, E * (int64_t)dm.n * dm.ld, E * (int64_t)dm.nu, E * (int64_t)dm.Nb * dm.m,
                   E * (int64_t)dm.nt, st);
  if (rc != IEDG_OK) return rc;
  rc = run_geometry(M, D->node_xyz, st);
  if (rc != IEDG_OK || !M->mass_scaled) return rc;
  // inverse Cholesky factors of the mass matrices for the scaled mixed forms
  CUDA_TRY(dalloc(M, &M->Linv32, (size_t)E * dm.Np * dm.Np));
  int flag = 0;
  CUDA_TRY(cudaMemsetAsync(M->dev_flag, 0, sizeof(int), st));
  CUDA_TRY(launch_mass_chol(M, st));
  CUDA_TRY(cudaMemcpyAsync(&flag, M->dev_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (flag) return fail(M, IEDG_ERR_MESH, "element mass matrix not positive definite");
  return IEDG_OK;
}

// Storage precision (FP64 or FP32 element matrices), the Schur GEMM's operands on the
// mixed path and the default LU form, the fastest measured on GB300: FP64 DFMA; FP32
// with FFMA updates on uniform meshes, with every trailing update on the tensor cores
// on meshes of mixed orders (the order-4 elements' long panels favour it).
static void set_precision(iedg_mesh* M, int precision, bool mixed_orders) {
  M->precision = precision == IEDG_PRECISION_FP64 ? 0 : 1;
  M->schur_in = precision == IEDG_PRECISION_MIXED_TF32   ? kSchurTf32
                : precision == IEDG_PRECISION_MIXED_BF16 ? kSchurBf16
                                                         : kSchurFp32;
  M->sched.lu_tensor = M->precision == 0 ? 0 : (M->schur_in != kSchurFp32 ? 1 : (mixed_orders ? 2 : 0));
}

static int check_desc(const iedg_mesh_desc* D, bool mixed) {
  iedg_mesh* M = nullptr;
  if (!(D->dim == 2 || D->dim == 3)) return fail(M, IEDG_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (!mixed && (D->order < 1 || D->order > (D->dim == 3 ? 4 : 3)))
    return fail(M, IEDG_ERR_UNSUPPORTED, "order must be 1..4 (3D) or 1..3 (2D)");
  if (D->quad_extra < 1 || D->quad_extra > 3)
    return fail(M, IEDG_ERR_UNSUPPORTED, "quad_extra must be 1..3");
  if (D->precision < IEDG_PRECISION_FP64 || D->precision > IEDG_PRECISION_MIXED_BF16)
    return fail(M, IEDG_ERR_UNSUPPORTED, "precision must be one of IEDG_PRECISION_FP64, _MIXED, _MIXED_TF32, _MIXED_BF16");
  if (D->stab != 0 && D->stab != 1)
    return fail(M, IEDG_ERR_UNSUPPORTED, "stab must be 0 (Lax-Friedrichs) or 1 (Roe-type)");
  if (D->n_elem <= 0 || D->n_trace <= 0 || !D->node_xyz || !D->elem_trace)
    return fail(M, IEDG_ERR_INVALID_ARG, "empty mesh or null mesh arrays");
  if (!(D->gamma > 1.0) || !(D->Pr > 0) || !(D->Re > 0) || !(D->alpha >= 0))
    return fail(M, IEDG_ERR_INVALID_ARG, "physical parameters out of range");
  if (D->flags & ~IEDG_FLAG_MASS_SCALING) return fail(M, IEDG_ERR_INVALID_ARG, "unknown descriptor flags");
  if ((D->flags & IEDG_FLAG_MASS_SCALING) && D->precision == IEDG_PRECISION_FP64)
    return fail(M, IEDG_ERR_INVALID_ARG, "mass-matrix scaling applies to the mixed forms only");
  if ((D->flags & IEDG_FLAG_MASS_SCALING) && mixed)
    return fail(M, IEDG_ERR_UNSUPPORTED, "mass-matrix scaling is not available on meshes with mixed orders");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(M, IEDG_ERR_CUDA, "no CUDA device");
  return IEDG_OK;
}

static void destroy_impl(iedg_mesh* M) {
  for (iedg_mesh* C : M->groups) destroy_impl(C);
  M->groups.clear();
  if (M->oz_scratch) cudaFree(M->oz_scratch);
  M->oz_scratch = nullptr;
  free_all(M);
  delete M;
}

extern "C" int iedg_create_mesh(const iedg_mesh_desc* D, void* stream, iedg_mesh** out) {
  iedg_mesh* M = nullptr;
  if (!D || !out) return fail(M, IEDG_ERR_INVALID_ARG, "null descriptor or output");
  *out = nullptr;
  int rc = check_desc(D, false);
  if (rc != IEDG_OK) return rc;
  M = new iedg_mesh();
  M->dm = make_dims(D->dim, D->order, D->quad_extra);
  M->ph = Phys{D->gamma, D->Pr, D->Re, D->alpha, D->stab, {0, 0, 0, 0, 0}};
  set_precision(M, D->precision, false);
  M->mass_scaled = (D->flags & IEDG_FLAG_MASS_SCALING) != 0;
  M->E = D->n_elem;
  M->T = D->n_trace;
  rc = create_impl(D, (cudaStream_t)stream, M);
  if (rc != IEDG_OK) {
    g_err = M->err;
    destroy_impl(M);
    return rc;
  }
  *out = M;
  return IEDG_OK;
}

// ------------------------------------------------------------------------------
// Meshes with mixed orders.  Internal element ids are grouped by order (ascending),
// user order kept within a group; one child handle per order holds that order's
// tables, the parent holds the trace space, the ragged element matrices (one buffer,
// per-element offset and leading dimension) and the per-element sizes.
// ------------------------------------------------------------------------------
template <class T>
static cudaError_t upload_to(iedg_mesh* M, const T** p, const std::vector<T>& h, cudaStream_t st) {
  T* q = nullptr;
  cudaError_t e = upload(M, &q, h, st);
  *p = q;
  return e;
}

static int create_mixed_impl(const iedg_mesh_desc* D, const int32_t* ord, const int32_t* fdeg,
                             const int32_t* fkind, cudaStream_t st, iedg_mesh* M) {
  const int d = D->dim, nf = 2 * d, m = d + 2;
  const int64_t E = M->E;
  const int pmax_allowed = d == 3 ? 4 : 3;
  M->mixed_orders = true;   // parent of per-order groups (set before its workspace is sized)
  for (int64_t e = 0; e < E; ++e) {
    if (ord[e] < 1 || ord[e] > pmax_allowed) return fail(M, IEDG_ERR_UNSUPPORTED, "element order out of range");
    for (int f = 0; f < nf; ++f) {
      if (fdeg[e * nf + f] < 0 || fdeg[e * nf + f] > 4)
        return fail(M, IEDG_ERR_UNSUPPORTED, "face degree must be 0 (continuous) or 1..4");
      if (fkind) {
        const int k = fkind[e * nf + f];
        if (k < kFaceInterior || k > kFaceWall) return fail(M, IEDG_ERR_INVALID_ARG, "face kind must be 0, 1 or 2");
        if (k != kFaceInterior && fdeg[e * nf + f] != ord[e])
          return fail(M, IEDG_ERR_INVALID_ARG, "a boundary face must carry private nodes of the element's degree");
      }
    }
  }
  std::vector<Dims> dmp(5);
  std::vector<HostRef> refs(5);
  std::vector<int> present;
  for (int p = 1; p <= 4; ++p)
    for (int64_t e = 0; e < E; ++e)
      if (ord[e] == p) { present.push_back(p); break; }
  for (int p : present) { dmp[p] = make_dims(d, p, D->quad_extra); refs[p] = build_reference(dmp[p]); }
  auto on_face = [&](int p, int a, int f) {
    int r = f / 2, v = a;
    for (int t = 0; t < r; ++t) v /= (p + 1);
    return (v % (p + 1)) == ((f % 2) ? p : 0);
  };
  // slot structure of every element (user order)
  std::vector<int> nbv(E);
  std::vector<int64_t> unode(E + 1, 0), uslot(E + 1, 0);
  for (int64_t e = 0; e < E; ++e) {
    const int p = ord[e];
    const Dims& dp = dmp[p];
    int cnt = 0;
    for (int a = 0; a < dp.Np; ++a) {
      if (refs[p].slot[a] < 0) continue;
      for (int f = 0; f < nf; ++f)
        if (fdeg[e * nf + f] == 0 && on_face(p, a, f)) { ++cnt; break; }
    }
    for (int f = 0; f < nf; ++f) {
      int q = fdeg[e * nf + f];
      if (q > 0) cnt += (d == 3 ? (q + 1) * (q + 1) : q + 1);
    }
    nbv[e] = cnt;
    unode[e + 1] = unode[e] + dp.Np;
    uslot[e + 1] = uslot[e] + cnt;
  }
  // internal ids: grouped by order
  M->perm.assign(E, 0);
  M->gstart.clear();
  std::vector<std::vector<int64_t>> gel;
  {
    int64_t next = 0;
    for (int p : present) {
      M->gstart.push_back(next);
      gel.emplace_back();
      for (int64_t e = 0; e < E; ++e)
        if (ord[e] == p) { M->perm[e] = next++; gel.back().push_back(e); }
    }
  }
  M->unode = unode;
  M->n_nodes = unode[E];
  int64_t P = 0;
  for (int64_t e = 0; e < E; ++e) P = std::max<int64_t>(P, nbv[e]);
  M->nb_pack = P;
  // per-element sizes in internal order
  std::vector<int> in_n(E), in_nu(E), in_ld(E), in_nb(E);
  std::vector<int64_t> in_soff(E), in_poff(E);
  for (int64_t e = 0; e < E; ++e) {
    const int64_t i = M->perm[e];
    const Dims& dp = dmp[ord[e]];
    in_nb[i] = nbv[e];
    in_nu[i] = dp.nu;
    in_n[i] = dp.nu + m * nbv[e];
    in_ld[i] = (in_n[i] + 1 + 3) & ~3;
  }
  int64_t S_total = 0, piv_total = 0;
  for (int64_t i = 0; i < E; ++i) {
    in_soff[i] = S_total;
    in_poff[i] = piv_total;
    S_total += (int64_t)in_n[i] * in_ld[i];
    piv_total += in_nu[i];
  }
  std::vector<int64_t> order(E);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return in_n[a] > in_n[b]; });
  // parent sizes: the largest of every kind (shared-memory sizing of the batched LU)
  Dims pd = dmp[present.back()];
  pd.Nb = (int)P;
  pd.nt = m * (int)P;
  pd.n = *std::max_element(in_n.begin(), in_n.end());
  pd.nu = *std::max_element(in_nu.begin(), in_nu.end());
  pd.ld = *std::max_element(in_ld.begin(), in_ld.end());
  M->dm = pd;
  // pattern and gather lists (user element order)
  {
    std::vector<const int64_t*> lists(E);
    std::vector<int> lens(E);
    std::vector<int64_t> ids(E);
    for (int64_t e = 0; e < E; ++e) { lists[e] = D->elem_trace + uslot[e]; lens[e] = nbv[e]; ids[e] = M->perm[e]; }
    int rc = setup_pattern(M, lists, lens, ids, P, st);
    if (rc != IEDG_OK) return rc;
  }
  // children
  std::vector<int64_t> rhat_off, re_off;
  int64_t rhat_total = 0, re_total = 0;
  for (size_t c = 0; c < present.size(); ++c) {
    const int p = present[c];
    iedg_mesh* C = new iedg_mesh();
    M->groups.push_back(C);
    Dims cd = dmp[p];
    int nbmax = 0;
    for (int64_t e : gel[c]) nbmax = std::max(nbmax, nbv[e]);
    cd.Nb = nbmax;
    cd.nt = m * nbmax;
    cd.n = cd.nu + cd.nt;
    cd.ld = (cd.n + 1 + 3) & ~3;
    C->dm = cd;
    C->ph = M->ph;
    C->precision = M->precision;
    C->schur_in = M->schur_in;
    C->E = (int64_t)gel[c].size();
    C->T = M->T;
    C->sched = M->sched;
    if (fkind)
      for (int64_t e : gel[c])
        for (int f = 0; f < nf; ++f)
          if (fkind[e * nf + f] != kFaceInterior) C->has_boundary = true;
    rhat_off.push_back(rhat_total);
    re_off.push_back(re_total);
    rhat_total += C->E * (int64_t)nbmax * m;
    re_total += C->E * (int64_t)nbmax * m;
  }
  // ragged sources of the R scatter, per-element LU sizes
  std::vector<int64_t> b_rhat(E), b_re(E), b_S(E);
  std::vector<int> ss_rhat(E, m), cs_rhat(E, 1), ss_re(E, 1), cs_re(E), ss_S(E), cs_S(E);
  for (size_t c = 0; c < present.size(); ++c) {
    const int Nbc = M->groups[c]->dm.Nb;
    for (int64_t k = 0; k < (int64_t)gel[c].size(); ++k) {
      const int64_t i = M->gstart[c] + k;
      b_rhat[i] = rhat_off[c] + k * (int64_t)Nbc * m;
      b_re[i] = re_off[c] + k * (int64_t)m * Nbc;
      cs_re[i] = Nbc;
      b_S[i] = in_soff[i] + (int64_t)in_nu[i] * in_ld[i] + in_n[i];
      ss_S[i] = in_ld[i];
      cs_S[i] = in_nb[i] * in_ld[i];
    }
  }
  int rc = alloc_owner(M, S_total, piv_total, rhat_total, re_total, st);
  if (rc != IEDG_OK) return rc;
  CUDA_TRY(upload_to(M, &M->lud.soff, in_soff, st));
  CUDA_TRY(upload_to(M, &M->lud.n, in_n, st));
  CUDA_TRY(upload_to(M, &M->lud.nu, in_nu, st));
  CUDA_TRY(upload_to(M, &M->lud.ld, in_ld, st));
  CUDA_TRY(upload_to(M, &M->lud.poff, in_poff, st));
  CUDA_TRY(upload_to(M, &M->lud.order, order, st));
  CUDA_TRY(upload_to(M, &M->el_nb, in_nb, st));
  CUDA_TRY(upload_to(M, &M->rs_rhat.base, b_rhat, st));
  CUDA_TRY(upload_to(M, &M->rs_rhat.ss, ss_rhat, st));
  CUDA_TRY(upload_to(M, &M->rs_rhat.cs, cs_rhat, st));
  CUDA_TRY(upload_to(M, &M->rs_re.base, b_re, st));
  CUDA_TRY(upload_to(M, &M->rs_re.ss, ss_re, st));
  CUDA_TRY(upload_to(M, &M->rs_re.cs, cs_re, st));
  CUDA_TRY(upload_to(M, &M->rs_S.base, b_S, st));
  CUDA_TRY(upload_to(M, &M->rs_S.ss, ss_S, st));
  CUDA_TRY(upload_to(M, &M->rs_S.cs, cs_S, st));
  CUDA_TRY(cudaStreamSynchronize(st));

  for (size_t c = 0; c < present.size(); ++c) {
    iedg_mesh* C = M->groups[c];
    const int p = present[c];
    const Dims& cd = C->dm;
    const HostRef& R = refs[p];
    const int64_t Ec = C->E;
    const int Nb = cd.Nb, Np = cd.Np, Nfq = cd.Nfq, Nfn = cd.Nfn, nq1 = cd.nq1;
    int NFS = Nfn;
    for (int64_t e : gel[c])
      for (int f = 0; f < nf; ++f) {
        int q = fdeg[e * nf + f];
        if (q > 0) NFS = std::max(NFS, d == 3 ? (q + 1) * (q + 1) : q + 1);
      }
    std::vector<int> t_nb(Ec), t_nfs(Ec * nf, 0), t_fs(Ec * nf * NFS, 0), t_fdeg(Ec * nf), t_sfl(Ec * Nb * 3, -1),
        t_kind(Ec * nf, 0);
    std::vector<double> t_muf((size_t)Ec * nf * Nfq * NFS, 0.0);
    std::vector<int64_t> t_et((size_t)Ec * Nb, 0), t_gnode(Ec);
    std::vector<double> X((size_t)Ec * Np * d);
    std::vector<int> eslot(Np);
    for (int64_t k = 0; k < Ec; ++k) {
      const int64_t e = gel[c][k];
      int cnt = 0;
      for (int a = 0; a < Np; ++a) {
        eslot[a] = -1;
        if (R.slot[a] < 0) continue;
        for (int f = 0; f < nf; ++f)
          if (fdeg[e * nf + f] == 0 && on_face(p, a, f)) { eslot[a] = cnt++; break; }
      }
      for (int f = 0; f < nf; ++f) {
        const int q = fdeg[e * nf + f];
        t_fdeg[k * nf + f] = q;
        t_kind[k * nf + f] = fkind ? fkind[e * nf + f] : kFaceInterior;
        int* fsf = &t_fs[((size_t)k * nf + f) * NFS];
        double* mu = &t_muf[((size_t)k * nf + f) * Nfq * NFS];
        if (q == 0) {
          t_nfs[k * nf + f] = Nfn;
          for (int tn = 0; tn < Nfn; ++tn) {
            const int a = R.fnode[f * Nfn + tn];
            fsf[tn] = eslot[a];
            for (int gf = 0; gf < Nfq; ++gf) mu[(size_t)gf * NFS + tn] = R.PhiF[(size_t)(f * Nfq + gf) * Np + a];
          }
        } else {
          const int q1 = q + 1, nq = d == 3 ? q1 * q1 : q1;
          t_nfs[k * nf + f] = nq;
          for (int j = 0; j < nq; ++j) {
            fsf[j] = cnt + j;
            const int j1 = j % q1, j2 = j / q1;
            for (int gf = 0; gf < Nfq; ++gf) {
              const int g1 = gf % nq1, g2 = gf / nq1;
              double v = R.LQ[((size_t)q * nq1 + g1) * 5 + j1];
              if (d == 3) v *= R.LQ[((size_t)q * nq1 + g2) * 5 + j2];
              mu[(size_t)gf * NFS + j] = v;
            }
          }
          cnt += nq;
        }
      }
      if (cnt != nbv[e]) return fail(M, IEDG_ERR_MESH, "inconsistent trace slot count");
      t_nb[k] = cnt;
      for (int f = 0; f < nf; ++f)
        for (int j = 0; j < t_nfs[k * nf + f]; ++j) {
          const int sl = t_fs[((size_t)k * nf + f) * NFS + j];
          if (sl < 0 || sl >= cnt) return fail(M, IEDG_ERR_MESH, "face node without a trace slot");
          int* fl = &t_sfl[((size_t)k * Nb + sl) * 3];
          int w = 0;
          while (w < 3 && fl[w] >= 0) ++w;
          if (w == 3) return fail(M, IEDG_ERR_MESH, "trace slot on more than three faces");
          fl[w] = f * NFS + j;
        }
      for (int s2 = 0; s2 < cnt; ++s2) t_et[(size_t)k * Nb + s2] = D->elem_trace[uslot[e] + s2];
      t_gnode[k] = unode[e];
      for (int i = 0; i < Np * d; ++i) X[(size_t)k * Np * d + i] = D->node_xyz[unode[e] * d + i];
    }
    TraceTab& tt = C->tt;
    tt.NFS = NFS;
    CUDA_TRY(upload_to(C, &tt.nb, t_nb, st));
    CUDA_TRY(upload_to(C, &tt.nfs, t_nfs, st));
    CUDA_TRY(upload_to(C, &tt.fs, t_fs, st));
    CUDA_TRY(upload_to(C, &tt.fdeg, t_fdeg, st));
    CUDA_TRY(upload_to(C, &tt.muf, t_muf, st));
    CUDA_TRY(upload_to(C, &tt.sfl, t_sfl, st));
    if (C->has_boundary) CUDA_TRY(upload_to(C, &tt.fkind, t_kind, st));
    CUDA_TRY(upload(C, &C->etrace, t_et, st));
    CUDA_TRY(upload(C, &C->gnode, t_gnode, st));
    tt.soff = M->lud.soff + M->gstart[c];
    tt.ldv = M->lud.ld + M->gstart[c];
    int rc2 = alloc_group(C, st);
    if (rc2 != IEDG_OK) return fail(M, rc2, C->err);
    if (M->precision == IEDG_PRECISION_MIXED) {
      float* m32 = nullptr;
      CUDA_TRY(dalloc(C, &m32, t_muf.size()));
      CUDA_TRY(launch_to_f32(tt.muf, m32, (int64_t)t_muf.size(), st));
      tt.muf32 = m32;
    }
    const size_t nod = (size_t)Ec * Np * m;
    CUDA_TRY(dalloc(C, &C->xu, nod));
    CUDA_TRY(dalloc(C, &C->xuref, nod));
    CUDA_TRY(dalloc(C, &C->xru, nod));
    CUDA_TRY(dalloc(C, &C->xq, nod * d));
    CUDA_TRY(dalloc(C, &C->xrq, nod * d));
    C->S = M->S;
    C->S32 = M->S32;
    C->piv = M->piv ? M->piv + in_poff[M->gstart[c]] : nullptr;
    C->pperm = M->pperm ? M->pperm + 3 * in_poff[M->gstart[c]] : nullptr;
    C->status = M->status + M->gstart[c];
    C->rhat = M->rhat + rhat_off[c];
    C->re64 = M->re64 + re_off[c];
    C->queue = M->queue;
    rc2 = run_geometry(C, X.data(), st);
    if (rc2 != IEDG_OK) return fail(M, rc2, C->err);
  }
  return IEDG_OK;
}

extern "C" int iedg_create_mesh_bc(const iedg_mesh_desc* D, const int32_t* elem_order, const int32_t* face_degree,
                                   const int32_t* face_kind, const double* u_far, void* stream, iedg_mesh** out) {
  iedg_mesh* M = nullptr;
  if (!D || !out || !elem_order || !face_degree) return fail(M, IEDG_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  int rc = check_desc(D, true);
  if (rc != IEDG_OK) return rc;
  const int nf = 2 * D->dim, m = D->dim + 2;
  bool farfield = false;
  if (face_kind)
    for (int64_t i = 0; i < D->n_elem * nf; ++i) farfield = farfield || face_kind[i] == kFaceFarField;
  if (farfield && !u_far) return fail(M, IEDG_ERR_INVALID_ARG, "far-field faces need the far-field state u_far");
  M = new iedg_mesh();
  M->ph = Phys{D->gamma, D->Pr, D->Re, D->alpha, D->stab, {0, 0, 0, 0, 0}};
  if (u_far)
    for (int i = 0; i < m; ++i) M->ph.ub[i] = u_far[i];
  set_precision(M, D->precision, true);
  M->E = D->n_elem;
  M->T = D->n_trace;
  rc = create_mixed_impl(D, elem_order, face_degree, face_kind, (cudaStream_t)stream, M);
  if (rc != IEDG_OK) {
    g_err = M->err;
    destroy_impl(M);
    return rc;
  }
  *out = M;
  return IEDG_OK;
}

extern "C" int iedg_create_mesh_mixed(const iedg_mesh_desc* D, const int32_t* elem_order,
                                      const int32_t* face_degree, void* stream, iedg_mesh** out) {
  return iedg_create_mesh_bc(D, elem_order, face_degree, nullptr, nullptr, stream, out);
}

extern "C" int iedg_element_sizes(const iedg_mesh* M, int32_t* Np, int32_t* Nb) {
  if (!M) return IEDG_ERR_INVALID_ARG;
  if (!M->mixed_orders) {
    for (int64_t e = 0; e < M->E; ++e) {
      if (Np) Np[e] = M->dm.Np;
      if (Nb) Nb[e] = M->dm.Nb;
    }
    return IEDG_OK;
  }
  std::vector<int> nb(M->E);
  if (Nb && cudaMemcpy(nb.data(), M->el_nb, M->E * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return IEDG_ERR_CUDA;
  for (int64_t e = 0; e < M->E; ++e) {
    if (Np) Np[e] = (int32_t)(M->unode[e + 1] - M->unode[e]);
    if (Nb) Nb[e] = nb[M->perm[e]];
  }
  return IEDG_OK;
}

// Compute entry points on meshes with mixed orders: each child runs the element
// kernels of its order on its own copies of the nodal arrays; the LU runs once over
// all elements (largest first) and the scatters read the ragged per-element results.
static int residual_mixed(iedg_mesh* M, const double* u, const double* uhat, const double* q, const double* u_ref,
                          double* q_out, double* r_q, double* r_u, double* r_fl, cudaStream_t st) {
  const int m = M->dm.m, d = M->dm.d;
  if (q && q_out)
    CUDA_TRY(cudaMemcpyAsync(q_out, q, M->n_nodes * m * d * sizeof(double), cudaMemcpyDeviceToDevice, st));
  for (iedg_mesh* C : M->groups) {
    CUDA_TRY(TRACED("nodal_in", launch_nodal_copy(C, m, u, C->xu, true, st)));
    if (q) CUDA_TRY(TRACED("nodal_in", launch_nodal_copy(C, m * d, q, C->xq, true, st)));
    if (u_ref) CUDA_TRY(TRACED("nodal_in", launch_nodal_copy(C, m, u_ref, C->xuref, true, st)));
    const double* ur = u_ref ? C->xuref : nullptr;
    if (!q) {
      CUDA_TRY(TRACED("lift", launch_lift(C, C->xu, uhat, C->xq, st)));
      if (q_out) CUDA_TRY(TRACED("nodal_out", launch_nodal_copy(C, m * d, C->xq, q_out, false, st)));
    }
    if (r_q) {
      if (q) CUDA_TRY(TRACED("lift", launch_lift(C, C->xu, uhat, C->qstar, st)));
      CUDA_TRY(TRACED("rq", launch_rq(C, C->xq, q ? C->qstar : C->xq, C->xrq, nullptr, st)));
      CUDA_TRY(TRACED("nodal_out", launch_nodal_copy(C, m * d, C->xrq, r_q, false, st)));
    }
    if (r_u || r_fl) {
      CUDA_TRY(TRACED("points_residual",
                      launch_points(C, C->xu, C->xq, nullptr, uhat, ur, false, r_u ? C->xru : nullptr, C->rhat, st)));
      if (r_u) CUDA_TRY(TRACED("nodal_out", launch_nodal_copy(C, m, C->xru, r_u, false, st)));
    }
  }
  if (r_fl) CUDA_TRY(TRACED("scatter_R", launch_scatter_R_ragged(M, M->rs_rhat, M->rhat, r_fl, st)));
  return IEDG_OK;
}

static int assemble_mixed(iedg_mesh* M, const double* u, const double* q, const double* uhat, const double* u_ref,
                          double* K, double* R, cudaStream_t st) {
  const int m = M->dm.m, d = M->dm.d;
  CUDA_TRY(cudaMemsetAsync(M->status, 0, M->E, st));
  for (iedg_mesh* C : M->groups) {
    CUDA_TRY(TRACED("nodal_in", launch_nodal_copy(C, m, u, C->xu, true, st)));
    CUDA_TRY(TRACED("nodal_in", launch_nodal_copy(C, m * d, q, C->xq, true, st)));
    if (u_ref) CUDA_TRY(TRACED("nodal_in", launch_nodal_copy(C, m, u_ref, C->xuref, true, st)));
    CUDA_TRY(TRACED("lift", launch_lift(C, C->xu, uhat, C->qstar, st)));
    CUDA_TRY(TRACED("rq", launch_rq(C, C->xq, C->qstar, nullptr, C->rhoq, st)));
    CUDA_TRY(TRACED("points_jacobian", launch_points(C, C->xu, C->xq, C->qstar, uhat, u_ref ? C->xuref : nullptr,
                                                     true, nullptr, nullptr, st)));
    if (assemble_sf_supported(C->dm))
      CUDA_TRY(TRACED("assemble", launch_assemble_sf(C, st)));
    else
      CUDA_TRY(TRACED("assemble", launch_assemble(C, st)));
  }
  CUDA_TRY(TRACED("lu_schur", launch_lu(M, st)));
  if (M->precision != IEDG_PRECISION_FP64) {
    for (iedg_mesh* C : M->groups) CUDA_TRY(TRACED("solve_prep", launch_solve_prep(C, st)));
    for (iedg_mesh* C : M->groups) CUDA_TRY(TRACED("refine", launch_refine(C, st)));
  }
  CUDA_TRY(TRACED("scatter_K", launch_scatter_K(M, K, st)));
  if (M->precision == IEDG_PRECISION_FP64)
    CUDA_TRY(TRACED("scatter_R", launch_scatter_R_ragged(M, M->rs_S, M->S, R, st)));
  else
    CUDA_TRY(TRACED("scatter_R", launch_scatter_R_ragged(M, M->rs_re, M->re64, R, st)));
  M->assembled = true;
  return IEDG_OK;
}

static int backsub_mixed_orders(iedg_mesh* M, const double* duhat, double* du, double* dq, cudaStream_t st) {
  const int m = M->dm.m, d = M->dm.d;
  for (iedg_mesh* C : M->groups) {
    if (M->precision == IEDG_PRECISION_FP64)
      CUDA_TRY(TRACED("backsub", launch_backsub(C, duhat, C->xru, C->xrq, st)));
    else
      CUDA_TRY(TRACED("backsub", launch_backsub_mixed(C, duhat, C->xru, C->xrq, st)));
    CUDA_TRY(TRACED("nodal_out", launch_nodal_copy(C, m, C->xru, du, false, st)));
    CUDA_TRY(TRACED("nodal_out", launch_nodal_copy(C, m * d, C->xrq, dq, false, st)));
  }
  return IEDG_OK;
}

extern "C" int iedg_destroy_mesh(iedg_mesh* M) {
  if (!M) return IEDG_ERR_INVALID_ARG;
  drain_events(M);
  destroy_impl(M);
  return IEDG_OK;
}

extern "C" int iedg_mesh_info(const iedg_mesh* M, int32_t* Np, int32_t* Nb, int64_t* nnzb,
                              int64_t* ws) {
  if (!M) return IEDG_ERR_INVALID_ARG;
  if (Np) *Np = M->dm.Np;
  if (Nb) *Nb = M->dm.Nb;
  if (nnzb) *nnzb = M->nnzb;
  if (ws) {
    *ws = M->ws_bytes;
    for (const iedg_mesh* C : M->groups) *ws += C->ws_bytes;
  }
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
  if (M->mixed_orders) return residual_mixed(M, u, uhat, q, u_ref, q_out, r_q, r_u, r_fl, st);
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
  if (M->mixed_orders) return assemble_mixed(M, u, q, uhat, u_ref, K, R, st);
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
  if (M->mass_scaled) CUDA_TRY(TRACED("mass_scale", launch_mass_scale(M, st)));
  if (M->fault.zero_row_elem >= 0) CUDA_TRY(TRACED("fault_zero_row", launch_zero_row(M, st)));
  CUDA_TRY(TRACED("lu_schur", launch_lu(M, st)));
  if (M->precision != IEDG_PRECISION_FP64) {
    CUDA_TRY(TRACED("solve_prep", launch_solve_prep(M, st)));
    CUDA_TRY(TRACED("refine", launch_refine(M, st)));
    CUDA_TRY(TRACED("fallback_fp64", launch_fallback(M, st)));
  }
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
  if (M->mixed_orders) return backsub_mixed_orders(M, duhat, du, dq, st);
  if (M->precision == IEDG_PRECISION_FP64) {
    CUDA_TRY(TRACED("backsub", launch_backsub(M, duhat, du, dq, st)));
  } else {
    CUDA_TRY(TRACED("backsub", launch_backsub_mixed(M, duhat, du, dq, st)));
    // elements condensed again in FP64 take their updates from the FP64 factors
    if (M->fb_S)
      CUDA_TRY(TRACED("backsub_fp64_fallback",
                      launch_backsub_list(M, M->fb_S, M->fb_list, kFallbackSlots, duhat, du, dq, st)));
  }
  return IEDG_OK;
}

extern "C" int64_t iedg_element_status(iedg_mesh* M, int8_t* out, void* stream) {
  if (!M || !out) return fail(M, IEDG_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (M->mixed_orders) {
    std::vector<int8_t> tmp(M->E);
    CUDA_TRY(cudaMemcpyAsync(tmp.data(), M->status, M->E, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t e = 0; e < M->E; ++e) out[e] = tmp[M->perm[e]];
  } else {
    CUDA_TRY(cudaMemcpyAsync(out, M->status, M->E, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
  }
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

extern "C" int iedg_set_fault_injection(iedg_mesh* M, const iedg_fault_injection* f) {
  if (!M || !f) return fail(M, IEDG_ERR_INVALID_ARG, "null argument");
  if (f->zero_row_elem < -1 || f->zero_row_elem >= M->E || f->refine_iters < -1 || f->refine_iters > 16 ||
      f->tc_wait_limit < -1 || (f->zero_row_elem >= 0 && (f->zero_row < 0 || f->zero_row >= M->dm.nu)))
    return fail(M, IEDG_ERR_INVALID_ARG, "fault injection values out of range");
  if (f->zero_row_elem >= 0 && M->mixed_orders)
    return fail(M, IEDG_ERR_UNSUPPORTED, "zero-row injection is only available on uniform meshes");
  M->fault.zero_row_elem = f->zero_row_elem;
  M->fault.zero_row = f->zero_row;
  M->fault.refine_iters = f->refine_iters;
  M->fault.tc_wait_limit = f->tc_wait_limit;
  for (iedg_mesh* C : M->groups) C->fault = M->fault;
  return IEDG_OK;
}

extern "C" int iedg_get_schedule(const iedg_mesh* M, iedg_schedule* out) {
  if (!M || !out) return IEDG_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->lu_persistent = M->sched.lu_persistent;
  out->lu_panel = M->sched.lu_panel;
  out->asm_chunk = M->sched.asm_chunk;
  out->lu_tensor = M->sched.lu_tensor;
  for (int i = 0; i < 4; ++i) out->asm_chunk_by_order[i] = M->sched.asm_chunk_by_order[i];
  return IEDG_OK;
}

extern "C" int iedg_set_schedule(iedg_mesh* M, const iedg_schedule* in) {
  if (!M || !in) return fail(M, IEDG_ERR_INVALID_ARG, "null argument");
  if ((in->lu_persistent != 0 && in->lu_persistent != 1) || (in->lu_panel != 16 && in->lu_panel != 32) ||
      (in->asm_chunk != 0 && in->asm_chunk != 8 && in->asm_chunk != 16 && in->asm_chunk != 32) ||
      (in->lu_tensor < 0 || in->lu_tensor > 2) || (in->lu_tensor == 2 && M->precision == IEDG_PRECISION_FP64))
    return fail(M, IEDG_ERR_INVALID_ARG, "schedule values out of range");
  for (int i = 0; i < 4; ++i) {
    const int c = in->asm_chunk_by_order[i];
    if (c != 0 && c != 8 && c != 16 && c != 32) return fail(M, IEDG_ERR_INVALID_ARG, "schedule values out of range");
  }
  if (M->precision == IEDG_PRECISION_FP64 && in->lu_tensor == 1) {
    // the FP64 tensor-core Schur form needs per-CTA slice buffers: allocated here, so
    // that compute calls allocate nothing
    const cudaError_t err = prepare_lu64_oz(M);
    if (err != cudaSuccess)
      return fail(M, err == cudaErrorMemoryAllocation ? IEDG_ERR_OOM : IEDG_ERR_CUDA,
                  std::string("FP64 tensor-core Schur buffers: ") + cudaGetErrorString(err));
  }
  M->sched.lu_persistent = in->lu_persistent;
  M->sched.lu_panel = in->lu_panel;
  M->sched.asm_chunk = in->asm_chunk;
  M->sched.lu_tensor = in->lu_tensor;
  for (int i = 0; i < 4; ++i) M->sched.asm_chunk_by_order[i] = in->asm_chunk_by_order[i];
  for (iedg_mesh* C : M->groups) {
    C->sched = M->sched;
    const int c = M->sched.asm_chunk_by_order[C->dm.p - 1];
    if (c) C->sched.asm_chunk = c;
  }
  return IEDG_OK;
}
