// Internal declarations of the IEDG sm_103a library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <string>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/iedg.h"

namespace iedg {

// Element sizes.  Local node a = a_0 + (p+1) a_1 + (p+1)^2 a_2, volume point g
// likewise over n_q1 Gauss points; face f = 2 r + side; face point fp = f Nfq + gf.
struct Dims {
  int d, p, m, np1, nq1;
  int Np, Nq, Nb, nf, Nfq, Nfp, Nfn;
  int nu;   // m Np   : element unknowns after q-elimination (u block)
  int nt;   // m Nb   : element trace unknowns
  int n;    // nu + nt: rows of the bordered element matrix
  int ld;   // leading dimension of the bordered matrix (>= n + 1, multiple of 4)
};

struct Phys {
  double gamma, Pr, Re, alpha;
  int stab;        // 0 = Lax-Friedrichs, 1 = Roe-type |A_n(uhat)|
  double ub[5];    // far-field state of far-field boundary faces
};

// face kinds of meshes with domain boundaries
constexpr int kFaceInterior = 0, kFaceFarField = 1, kFaceWall = 2;
// operands of the Schur GEMM K = D - W Z on the mixed path
constexpr int kSchurFp32 = 0, kSchurTf32 = 1, kSchurBf16 = 2;

// Launch schedule (host-side choices the autotuner sweeps; see iedg_schedule).
struct Schedule {
  int lu_persistent = 1;     // batched LU as a persistent grid with an element queue
  int lu_panel = 16;         // FP64 LU panel width (16 or 32; 32 only when it fits shared memory)
  int asm_chunk = 0;         // assembly column chunk (0 = default: 8 for FP64, 16 for FP32)
  int lu_tensor = 1;         // 0 = DFMA / FFMA updates; 1 = deferred Schur complement on tcgen05;
                             // 2 (mixed FP32 form) = every trailing update on tcgen05 (3xTF32)
  int asm_chunk_by_order[4] = {0, 0, 0, 0};   // mixed orders: chunk per order (0 = asm_chunk)
};

// Failure injection for tests (iedg_set_fault_injection).
struct Fault {
  int64_t zero_row_elem = -1;   // element (internal id) whose u-row zero_row is zeroed before the LU
  int zero_row = 0;
  int refine_iters = -1;        // correction steps of the refinement (-1 = kRefineMaxIter)
  int tc_wait_limit = 0;        // polls of a tensor-core completion wait (0 = kTcWaitLimit, -1 = none)
};
constexpr int kTcWaitLimit = 1 << 26;

// Reference-element tables (device), shared by all elements.
struct RefTables {
  double* Phi;    // [Nq][Np]
  double* Dxi;    // [d][Nq][Np]
  double* Wq;     // [Nq]
  double* PhiF;   // [Nfp][Np]
  double* DxiF;   // [d][Nfp][Np]
  double* Wf;     // [Nfq]
  int* bnode;     // [Nb]   local node of trace slot s
  int* slot;      // [Np]   trace slot of node a, -1 for interior nodes
  int* fnode;     // [nf][Nfn] nodes of each face
  double* L1;     // [nq1][np1] 1D Lagrange basis at the 1D Gauss points
  double* dL1;    // [nq1][np1] its derivative
  double* LQ;     // [5][nq1][5] degree-q Gauss-Lobatto Lagrange basis at the 1D Gauss points
                  //              (private face nodes of meshes with mixed orders)
  float* LQ32;
  float* Phi32;   // FP32 copies for the mixed path (FP64 -> FP32 conversion is slow on GB300)
  float* Dxi32;
  float* PhiF32;
};

// Per-element geometry (device).
struct Geo {
  double* wdet;   // [E][Nq]          W_g detJ
  double* Jinv;   // [E][Nq][d][d]    Jinv[r][j] = d xi_r / d x_j
  double* fw;     // [E][Nfp]         W_f |cof(J) nref|
  double* fn;     // [E][Nfp][d]      unit outward normal
  double* Mass;   // [E][Np][Np]
  double* Gl;     // [E][d][Np][Np]   M^-1 B_l
  double* Hl;     // [E][d][Np][Nb]   M^-1 E_l
  double* GlV;    // [E][d][Nq][Np]   Phi Gl   (lifting at volume points)
  double* HlV;    // [E][d][Nq][Nb]
  double* GlF;    // [E][d][Nfp][Np]  PhiF Gl  (lifting at face points)
  double* HlF;    // [E][d][Nfp][Nb]
  // FP32 copies (mixed path only)
  float *Mass32, *GlV32, *HlV32, *GlF32, *HlF32;
};

// Point tables written by the point kernel for the assembly kernel.
struct PointJac {
  double* Jv;     // [E][m][m][(1+d) d][Nq]: c<d: cu_r ; c = d + l d + r: cq_lr  (w Jinv folded)
  double* Jf;     // [E][m][m][1+d][Nfp]   : c=0: wf dfhat/duhat ; c=1+l: wf dfhat/dq_l
  double* lamw;   // [E][Nfp]              : wf lambda  (dfhat/du = lambda I, Lax-Friedrichs)
  double* Su;     // [E][m][m][Nfp]        : wf dfhat_i/du_k = wf S_ik (Roe-type only, else null)
  double* Jb;     // [E][m][m][2+d][Nfp]   : boundary faces only: wf dbhat/duhat, wf dbhat/du,
                  //                          wf dbhat/dq_l (null without boundary faces)
  float *Jv32, *Jf32, *lamw32, *Su32, *Jb32;   // FP32 copies written by the point kernel (mixed path only)
};

// Per-element trace description of meshes with mixed orders.  A face shared with an
// element of the same order carries the continuous trace of the uniform case (the
// element basis restricted to the face, slots = its boundary nodes on such faces); a
// face shared with another order carries (q+1)^(d-1) private nodes of degree q at the
// Gauss-Lobatto points of the face (first tangential direction fastest).  All pointers
// are null for uniform meshes.
struct TraceTab {
  const int* nb = nullptr;         // [E] trace slots of each element (<= Dims.Nb)
  const int* nfs = nullptr;        // [E][nf] slots whose basis function is nonzero on each face
  const int* fs = nullptr;         // [E][nf][NFS] those slots (continuous face: in face-node order)
  const int* fdeg = nullptr;       // [E][nf] 0 = continuous face, q = private nodes of degree q
  const double* muf = nullptr;     // [E][nf][Nfq][NFS] their values at the face points
  const float* muf32 = nullptr;
  const int* sfl = nullptr;        // [E][Nb][3] faces of each slot, f NFS + j (-1 = none)
  const int* fkind = nullptr;      // [E][nf] kFace* (null: no domain boundary)
  const int64_t* soff = nullptr;   // [E] offset of the element's bordered matrix in S
  const int* ldv = nullptr;        // [E] its leading dimension
  int NFS = 0;
};

// Per-element sizes of the batched LU (null pointers: every element has the sizes of
// Dims and sits at e n ld).  order lists the elements in the order the persistent
// grid takes them (largest first).
struct LuDesc {
  const int64_t* soff = nullptr;
  const int* n = nullptr;
  const int* nu = nullptr;
  const int* ld = nullptr;
  const int64_t* poff = nullptr;   // pivot offsets (mixed path)
  const int64_t* order = nullptr;
};

// Location of the per-slot values of a ragged source: value (e, s, i) at
// base[e] + s ss[e] + i cs[e].
struct RaggedSrc {
  const int64_t* base = nullptr;
  const int* ss = nullptr;
  const int* cs = nullptr;
};

// Tables of one precision for the assembly kernels (the FP32 set is converted once
// per mesh / per point pass, so no FP64 value is touched on the FP32 path).
template <class T>
struct AsmTab {
  const T *Phi, *Dxi, *PhiF;
  const T *Jv, *Jf, *lamw, *Su, *Jb;
  const T *GlV, *HlV, *GlF, *HlF, *Mass;
};

}  // namespace iedg

struct iedg_mesh {
  iedg::Dims dm;
  iedg::Phys ph;
  int64_t E = 0, T = 0, nnzb = 0;
  int64_t max_row_blocks = 0;   // longest block row of K (blocks)
  iedg::RefTables ref{};
  iedg::Geo geo{};
  iedg::PointJac pj{};
  int64_t* etrace = nullptr;    // [E][Nb]
  int64_t* row_ptr = nullptr;   // [T+1]
  int32_t* col = nullptr;       // [nnzb]
  int64_t* kc_ptr = nullptr;    // [nnzb+1] gather list of K blocks
  int64_t* kc_src = nullptr;    //   e Nb^2 + s Nb + t
  int64_t* rc_ptr = nullptr;    // [T+1]    gather list of trace rows
  int64_t* rc_src = nullptr;    //   e Nb + s
  double* qstar = nullptr;      // [E][Np][m][d] lifted gradient (R_q = 0)
  double* rhoq = nullptr;       // [E][Np][m][d] q - qstar of the last assembly
  double* rhat = nullptr;       // [E][Nb][m]    element trace residuals
  double* S = nullptr;          // [E][n][ld]    bordered element matrices (FP64 path)
  // mixed path (FP32 condensation, FP64 refinement)
  int precision = 0;            // 0 = FP64, 1 = mixed (FP32 element matrix and LU)
  int schur_in = 0;             // mixed: operands of the Schur GEMM (kSchurFp32 / Tf32 / Bf16)
  float* S32 = nullptr;         // [E][n][ld]    bordered element matrices, FP32, L kept
  bool mass_scaled = false;     // mixed forms: element systems scaled by the mass matrix (iedg_mass_scale.cu)
  float* Linv32 = nullptr;      // [E][Np][Np]   inverse Cholesky factor of the mass matrix, FP32
  int* piv = nullptr;           // [E][nu]       pivot rows of the FP32 partial LU
  int* pperm = nullptr;         // [E][3 nu]     each panel's interchanges composed (iedg_refine.cu)
  double* rhs64 = nullptr;      // [E][n]        FP64 right-hand sides F~, G~
  double* y64 = nullptr;        // [E][nu]       refined A~^-1 F~
  double* re64 = nullptr;       // [E][m][Nb]    refined R_e (component-major)
  int8_t* status = nullptr;     // [E]
  // FP64 fallback of the mixed forms (uniform meshes): kFallbackSlots FP64 element
  // matrices and the slot bookkeeping (iedg_fallback.cu)
  double* fb_S = nullptr;       // [slots][n][ld]
  int64_t* fb_list = nullptr;   // [slots] element of each slot, -1 = empty
  int* fb_slot = nullptr;       // [E]     slot of each element, -1 = none
  int8_t* fb_status = nullptr;  // [slots] status of the FP64 partial LU
  int* fb_count = nullptr;      // slots in use
  int64_t* queue = nullptr;     // element counter of persistent launches
  float* oz_scratch = nullptr;  // FP64 tensor-core Schur form: per-CTA slice buffers (freed with the handle)
  unsigned oz_grid = 0;
  // meshes with mixed orders: the parent handle holds the trace space, the ragged
  // element matrices and the per-element sizes; one child handle per order holds the
  // element tables of that order (internal element ids are grouped by order)
  iedg::TraceTab tt;            // child: trace description of its elements
  bool has_boundary = false;    // child: some element has a domain-boundary face
  bool mixed_orders = false;    // parent
  std::vector<iedg_mesh*> groups;
  std::vector<int64_t> gstart;  // parent: first internal id of each group
  std::vector<int64_t> perm;    // parent: internal id of each user element
  std::vector<int64_t> unode;   // parent: user node offset of each user element [E+1]
  int64_t n_nodes = 0;          // parent: nodes of all elements
  int64_t nb_pack = 0;          // parent: slot stride of the packed (e, s) gather entries
  iedg::LuDesc lud;             // parent
  iedg::RaggedSrc rs_rhat, rs_S, rs_re;   // parent: sources of the R scatter
  const int* el_nb = nullptr;   // parent: [E] trace slots per element (internal order)
  int64_t* gnode = nullptr;     // child: [E] user node offset of each element
  double *xu = nullptr, *xuref = nullptr, *xq = nullptr, *xru = nullptr, *xrq = nullptr;  // child nodal buffers
  // trace solve preconditioner: BILU(0) in multicolour order (built on first use)
  int prec_kind = 0;            // IEDG_PREC_BLOCK_JACOBI or IEDG_PREC_BILU0
  double* bf = nullptr;         // BILU(0) factors [nnzb][m][m]
  int64_t* brows = nullptr;     // [T] trace nodes sorted by (colour, index)
  std::vector<int64_t> bcptr;   // colour boundaries in brows
  double* kst = nullptr;        // trace solve: GMRES state on the device (Hessenberg, rotations, scalars)
  int32_t* bord = nullptr;      // [nnzb] per row: entry offsets in elimination order
  int32_t* bnlow = nullptr;     // [T] entries of each row ranked before the row
  std::vector<int32_t> bcolor;  // host: colour of every trace node
  double* kry = nullptr;        // trace solve: Krylov basis [IEDG_MAX_RESTART+1][T m] + 2 work vectors
  double* dinv = nullptr;       // trace solve: inverted diagonal blocks [T][m][m]
  double* kpart = nullptr;      // trace solve: dot-product partial sums
  double* khdev = nullptr;      // trace solve: small vector of coefficients
  iedg::Schedule sched;
  iedg::Fault fault;
  int* dev_flag = nullptr;      // geometry error flag
  bool assembled = false;
  // tracing: launches per kernel, events while profiling is on
  bool profiling = false;
  std::vector<std::string> kname;
  std::vector<int64_t> klaunch;
  std::vector<double> kms;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> kev;
  int64_t ws_bytes = 0;
  std::string err;
  std::vector<void*> allocs;
};

namespace iedg {

inline int idiv_up(int a, int b) { return (a + b - 1) / b; }

// kernels (launchers)
cudaError_t launch_geometry(iedg_mesh* M, const double* X, double* scratch, cudaStream_t st);
cudaError_t launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t st);
cudaError_t launch_lift(iedg_mesh* M, const double* u, const double* uhat, double* qstar, cudaStream_t st);
cudaError_t launch_points(iedg_mesh* M, const double* u, const double* q, const double* qs,
                          const double* uhat, const double* u_ref, bool jacobians,
                          double* r_u, double* rhat, cudaStream_t st);
cudaError_t launch_rq(iedg_mesh* M, const double* q, const double* qs, double* r_q, double* rhoq,
                      cudaStream_t st);
cudaError_t launch_assemble(iedg_mesh* M, cudaStream_t st);
cudaError_t launch_assemble_sf(iedg_mesh* M, cudaStream_t st);   // 3D, sum-factorised
bool assemble_sf_supported(const Dims& dm);
AsmTab<double> tables64(const iedg_mesh* M);
AsmTab<float> tables32(const iedg_mesh* M);
cudaError_t launch_lu(iedg_mesh* M, cudaStream_t st);
cudaError_t prepare_lu64_oz(iedg_mesh* M);   // slice buffers of the FP64 tensor-core Schur form
cudaError_t launch_lu32_mma(iedg_mesh* M, int n_max, cudaStream_t st);   // FP32 LU, tcgen05 trailing updates
cudaError_t launch_scatter_K(iedg_mesh* M, double* K, cudaStream_t st);
cudaError_t launch_scatter_R_ragged(iedg_mesh* M, const RaggedSrc& src, const double* base, double* R,
                                    cudaStream_t st);
// nodal arrays of a child: user layout [nodes][w] <-> child layout [E][Np][w]
cudaError_t launch_nodal_copy(iedg_mesh* C, int w, const double* src, double* dst, bool to_child,
                              cudaStream_t st);
cudaError_t launch_scatter_R(iedg_mesh* M, const double* src, int64_t src_elem_stride,
                             int64_t src_slot_stride, int64_t src_comp_stride, double* R,
                             cudaStream_t st);
cudaError_t launch_backsub(iedg_mesh* M, const double* duhat, double* du, double* dq,
                           cudaStream_t st);
cudaError_t launch_solve_prep(iedg_mesh* M, cudaStream_t st);
cudaError_t launch_refine(iedg_mesh* M, cudaStream_t st);
// FP64 fallback of flagged elements on the mixed path (iedg_fallback.cu)
constexpr int kFallbackSlots = 32;
cudaError_t launch_fallback(iedg_mesh* M, cudaStream_t st);
cudaError_t launch_assemble_list(iedg_mesh* M, double* S, const int64_t* elist, int64_t n_slots, cudaStream_t st);
cudaError_t launch_assemble_sf_list(iedg_mesh* M, double* S, const int64_t* elist, int64_t n_slots, cudaStream_t st);
cudaError_t launch_lu64_list(iedg_mesh* M, double* S, int64_t n_slots, const int64_t* active, int8_t* status,
                             cudaStream_t st);
cudaError_t launch_zero_row_fallback(iedg_mesh* M, cudaStream_t st);
cudaError_t launch_backsub_list(iedg_mesh* M, const double* S, const int64_t* elist, int64_t n_slots,
                                const double* duhat, double* du, double* dq, cudaStream_t st);
cudaError_t launch_zero_row(iedg_mesh* M, cudaStream_t st);   // Fault.zero_row_elem
cudaError_t launch_mass_chol(iedg_mesh* M, cudaStream_t st);   // L^-1 of the mass matrices (once per mesh)
cudaError_t launch_mass_scale(iedg_mesh* M, cudaStream_t st);  // S A~ S^T, S B~, C~ S^T of the FP32 systems
cudaError_t launch_backsub_mixed(iedg_mesh* M, const double* duhat, double* du, double* dq,
                                 cudaStream_t st);

inline int refine_iters(const iedg_mesh* M) { return M->fault.refine_iters >= 0 ? M->fault.refine_iters : 8; }
inline int tc_wait_limit(const iedg_mesh* M) {
  return M->fault.tc_wait_limit > 0 ? M->fault.tc_wait_limit : (M->fault.tc_wait_limit < 0 ? 0 : kTcWaitLimit);
}

// refinement controls of the mixed path
constexpr int kRefineMaxIter = 8;
constexpr double kRefineTol = 1e-14;      // stop at |r|_inf <= tol * |rhs|_inf
constexpr double kRefineFlag = 1e-10;     // flag the element if not reached

}  // namespace iedg
