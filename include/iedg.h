/*
 * iedg.h -- C ABI of the GB300 (sm_103a) IEDG local-problem library.
 *
 * The library implements the element-local part of every Newton step of the
 * Interior Embedded Discontinuous Galerkin (IEDG) discretisation of the
 * compressible Navier-Stokes equations (Fernandez, Nguyen, Roca, Peraire,
 * arXiv:1605.01020):
 *   - the residuals R_NS = (R_q, R_u) and R_FL of the weak form (Eq. IEDG a-c,
 *     Eq. NLS), with the Lax-Friedrichs or Roe-type numerical flux of Eq. IEDG (d);
 *   - the element blocks of the Newton matrix [A B; C D] and right-hand side
 *     [F; G] (Sec. 2.2.1), statically condensed onto the trace unknowns,
 *     K = D - C A^-1 B and R = G - C A^-1 F (Eq. LS), and assembled into a
 *     block compressed-row matrix with m x m blocks (Sec. 2.2.2);
 *   - the back-substitution dZ = A^-1 (F - B dU) after the trace solve.
 *
 * Conventions (all of them, including the readings where the paper is silent):
 *   d = 2 or 3, m = d + 2 conserved variables u = (rho, rho v_j, rho E).
 *   Elements are tensor-product quads/hexes of uniform degree p (1..4 in 3D,
 *   1..3 in 2D); local nodes are the Gauss-Lobatto-Legendre lattice, numbered
 *   lexicographically with the first reference direction fastest; Np = (p+1)^d.
 *   Trace slots of an element are its boundary nodes in that same order; Nb =
 *   (p+1)^d - (p-1)^d.  elem_trace[e][s] is the global trace node of slot s.
 *   The trace is continuous wherever two slots map to the same trace node (the
 *   EDG faces of the IEDG method, Sec. 2.1); periodic faces are ordinary interior
 *   faces.
 *   Quadrature: Gauss-Legendre with n_q1 = p + quad_extra points per direction.
 *   Physics: gamma, Pr, Re as in Sec. 2.1; temperature read as the specific
 *   internal energy e = E - |v|^2/2 and heat flux -(gamma/(Re Pr)) grad e
 *   (dissipative sign).  Implicit stage: R_u gains alpha M (u - u_ref), alpha =
 *   1 / (a_ii dt) of the DIRK stage (alpha = 0: steady).
 *   Newton signs: F = -R_NS, G = -R_FL, so K dU = R gives the Newton increment.
 *
 * Memory: every array argument of the compute calls is a DEVICE pointer owned by
 * the caller, in the layouts stated below (row-major, FP64), used on `stream`
 * (a cudaStream_t, NULL = legacy default stream).  The handle owns only its own
 * device workspace, allocated once in iedg_create_mesh.  Compute calls allocate
 * nothing and do not synchronise the host; kernel-side problems (zero pivot,
 * non-finite values) are recorded per element and read with iedg_element_status.
 * There is no CPU fallback: without a usable CUDA device calls return
 * IEDG_ERR_CUDA.  One handle must not be used from two streams at once.
 *
 * Errors: functions return IEDG_OK (0) or a negative code; the message of the
 * last failure is iedg_last_error(handle) (or iedg_last_error(NULL) for failures
 * before a handle exists).  No C++ exception crosses this interface.
 */
#ifndef IEDG_H
#define IEDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IEDG_OK                 0
#define IEDG_ERR_INVALID_ARG   -1
#define IEDG_ERR_CUDA          -2
#define IEDG_ERR_OOM           -3
#define IEDG_ERR_MESH          -4   /* detJ <= 0 somewhere, or bad element->trace map */
#define IEDG_ERR_NOT_ASSEMBLED -5   /* back-substitution before any assembly          */
#define IEDG_ERR_UNSUPPORTED   -6   /* valid request this build does not implement    */

/* element status codes (iedg_element_status) */
#define IEDG_ELEM_OK        0
#define IEDG_ELEM_REFINE    1   /* mixed path: refinement did not reach 1e-10 relative residual */
#define IEDG_ELEM_SINGULAR  2   /* exact zero pivot in the element block          */
#define IEDG_ELEM_NONFINITE 3   /* NaN/Inf met among the element's pivot candidates
                                   or in its Schur complement                      */
#define IEDG_ELEM_TIMEOUT   4   /* tensor-core forms: a bounded completion wait gave up
                                   (see iedg_set_fault_injection); the element was not
                                   factored                                         */
#define IEDG_ELEM_FALLBACK  5   /* mixed forms: the element's refinement did not reach
                                   1e-10, its tensor-core wait gave up or its FP32 LU
                                   met a zero pivot, and it was condensed again in FP64
                                   in the same call (K_e, R_e and its updates are the
                                   FP64 path's).  At most 32 elements per call, lowest
                                   ids first, get this; the others keep their flag.
                                   Uniform meshes only.                              */

#define IEDG_PRECISION_FP64  0   /* every step in FP64                                   */
#define IEDG_PRECISION_MIXED 1   /* element matrix and partial LU in FP32 (K to FP32
                                    accuracy); residuals, point Jacobians and the
                                    right-hand side R and updates du, dq refined to FP64 */
#define IEDG_PRECISION_MIXED_TF32 2  /* as MIXED, with the Schur complement K = D~ - W Z of
                                    the partial LU (W, Z the eliminated trace rows and the
                                    u-rows' trace columns) on the tensor cores with the
                                    operands rounded to TF32 and FP32 accumulation: K to
                                    TF32 accuracy; R, du, dq refined to FP64 as in MIXED   */
#define IEDG_PRECISION_MIXED_BF16 3  /* same with BF16 operands: K to BF16 accuracy        */

typedef struct iedg_mesh iedg_mesh;   /* opaque */

typedef struct {
  int32_t dim;              /* 2 or 3                                                */
  int32_t order;            /* polynomial degree p = k of approximation and geometry */
  int32_t quad_extra;       /* n_q1 = p + quad_extra Gauss points per direction (2)  */
  int32_t precision;        /* IEDG_PRECISION_FP64, _MIXED, _MIXED_TF32, _MIXED_BF16   */
  int64_t n_elem;
  int64_t n_trace;
  const double*  node_xyz;   /* HOST [n_elem][Np][dim]: isoparametric nodes (Sec. 3.1) */
  const int64_t* elem_trace; /* HOST [n_elem][Nb]: global trace node of each slot      */
  double gamma, Pr, Re, Minf, alpha;
  int32_t stab;             /* stabilisation S of Eq. IEDG d, evaluated at uhat:
                               0 = Lax-Friedrichs, S = (|vhat.n| + chat) I;
                               1 = Roe-type, S = |A_n(uhat)|, A_n the normal Jacobian of
                               the Euler flux (the absolute values of its eigenvalues
                               v_n, v_n +- c in its eigenbasis); both fully linearised,
                               d|x|/dx = sign(x) with sign(0) = 0                        */
  int32_t flags;            /* IEDG_FLAG_* (0 = none)                                */
} iedg_mesh_desc;

/* Mixed forms (precision 1-3, uniform meshes): before the FP32 partial LU the element
 * system is scaled by the element mass matrix M = L L^T (Cholesky): the u-block A~
 * becomes S A~ S^T, B~ becomes S B~ and C~ becomes C~ S^T with S = I_m (x) L^-1 (one
 * block per conserved component).  K and R are the same in exact arithmetic (Eq. LS
 * is invariant under this scaling); the scaled u-block is far better conditioned (the
 * implicit stage's alpha M becomes alpha I), and the TF32 / BF16 Schur operands W, Z
 * are those of the scaled system.  The refinement and back-substitution solve with
 * the scaled factors (x = S^T (S A~ S^T)^-1 S b).  No counterpart in the paper, which
 * has no precision discussion: the reading of "scaling by the element mass matrix".
 * IEDG_ERR_INVALID_ARG with FP64 handles, IEDG_ERR_UNSUPPORTED with mixed orders. */
#define IEDG_FLAG_MASS_SCALING 1

/* Builds the handle: copies the mesh to the device, computes per-element geometry
 * (Jacobians, weights, normals, mass matrix and the lifting operators of Eq. IEDG a)
 * on `stream`, builds the trace-matrix pattern and the gather lists, and allocates
 * all workspace.  Synchronises `stream` before returning.  IEDG_ERR_MESH if any
 * quadrature point has detJ <= 0 or a trace id is out of range. */
int iedg_create_mesh(const iedg_mesh_desc* desc, void* stream, iedg_mesh** out);

/* Meshes with mixed polynomial orders (no counterpart in the paper, which uses one
 * degree k per mesh; this is the trace sharing of Sec. 2.1 extended to elements of
 * different degrees).  Element e has degree elem_order[e] (HOST int32 [n_elem],
 * 1..4 in 3D, 1..3 in 2D; desc->order is ignored) and face_degree[e][f] (HOST int32
 * [n_elem][2 dim], faces f = 2 r + side in the order -x, +x, -y, +y, -z, +z):
 *   0      the face is shared with an element of the same degree and carries the
 *          continuous (EDG) trace of the uniform case;
 *   q > 0  the face carries (q+1)^(dim-1) private trace nodes, the Gauss-Lobatto
 *          points of degree q in the face's tangential reference coordinates (first
 *          tangential direction fastest) with the degree-q Lagrange basis; both
 *          neighbours list the same nodes (q = max of the two degrees in the
 *          workloads of this project).
 * The slots of element e: its boundary nodes that lie on at least one face with
 * face_degree 0 (lexicographic), then the private nodes of each other face in face
 * order; nb_e of them.  Every element-indexed array is RAGGED, elements in user order
 * with their own sizes, no padding: node_xyz [sum Np_e][dim], elem_trace [sum nb_e];
 * in the compute calls u, u_ref, r_u, du are [sum Np_e][m] and q, q_out, r_q, dq
 * [sum Np_e][m][dim].  K, R, uhat, duhat are as for uniform meshes.  The element
 * sizes are returned by iedg_element_sizes.  iedg_eval_residual_static returns
 * IEDG_ERR_UNSUPPORTED on such meshes; every other call works unchanged. */
int iedg_create_mesh_mixed(const iedg_mesh_desc* desc, const int32_t* elem_order,
                           const int32_t* face_degree, void* stream, iedg_mesh** out);

/* Meshes with domain boundaries (Sec. 2.1: the IEDG trace is continuous on interior
 * faces and discontinuous on boundary faces).  As iedg_create_mesh_mixed, plus
 * face_kind (HOST int32 [n_elem][2 dim], NULL = every face interior):
 *   0  interior face (shared with the neighbour, as above);
 *   1  far field (inflow / outflow): the trace equation on the face takes
 *      bhat = (A_n + |A_n|)/2 (uhat - u) + (A_n - |A_n|)/2 (uhat - u_far), A_n the
 *      normal Jacobian of the Euler flux and |A_n| its absolute value, both at uhat;
 *   2  no-slip adiabatic wall: bhat = (rhohat - rho, rho vhat, fhat_E), i.e. the trace
 *      density follows the interior, the trace velocity vanishes and the energy row of
 *      the numerical flux (the normal heat flux at a no-slip wall) is zero.
 * A boundary face must have face_degree equal to the element's order (its private
 * trace nodes belong to this element alone).  u_far (HOST double [m]) is required
 * when some face is a far-field face.  The element equations use the numerical flux
 * fhat on every face. */
int iedg_create_mesh_bc(const iedg_mesh_desc* desc, const int32_t* elem_order, const int32_t* face_degree,
                        const int32_t* face_kind, const double* u_far, void* stream, iedg_mesh** out);

/* Per-element node and trace-slot counts, HOST int32 [n_elem] each (either may be
 * NULL); for uniform meshes every entry is Np, Nb. */
int iedg_element_sizes(const iedg_mesh* mesh, int32_t* Np, int32_t* Nb);

int iedg_destroy_mesh(iedg_mesh* mesh);
const char* iedg_last_error(const iedg_mesh* mesh);

/* Sizes: Np, Nb, number of trace-matrix blocks nnzb (m x m each), bytes of device
 * workspace held by the handle.  Any output pointer may be NULL.  Meshes with mixed
 * orders report the largest Np and nb_e. */
int iedg_mesh_info(const iedg_mesh* mesh, int32_t* Np, int32_t* Nb, int64_t* nnzb,
                   int64_t* workspace_bytes);

/* Block compressed-row pattern of K (Sec. 2.2.2): one block row per trace node,
 * one block for every pair of trace nodes sharing an element, columns sorted
 * ascending.  Copies into caller DEVICE buffers row_ptr[n_trace+1], col[nnzb]. */
int iedg_trace_pattern(const iedg_mesh* mesh, int64_t* row_ptr, int32_t* col, void* stream);

/* Residual of Eq. IEDG (a)-(c).
 *   u    [n_elem][Np][m]      element states
 *   uhat [n_trace][m]         trace state
 *   q    [n_elem][Np][m][d]   gradient state q_ij = du_i/dx_j, or NULL: then q is
 *                             taken from R_q = 0 (local lifting of (u, uhat)) and
 *                             written to q_out (required in that case)
 *   u_ref [n_elem][Np][m] or NULL (= u): reference state of the implicit stage
 * Outputs (any may be NULL except that q_out is needed when q is NULL):
 *   r_q  [n_elem][Np][m][d], r_u [n_elem][Np][m], r_fl [n_trace][m] (overwritten). */
int iedg_eval_residual(iedg_mesh* mesh, const double* u, const double* uhat,
                       const double* q, const double* u_ref, double* q_out,
                       double* r_q, double* r_u, double* r_fl, void* stream);

/* One Newton linearisation, condensed (Sec. 2.2.1, Eq. LS):
 *   K_bsr [nnzb][m][m] values of K in the pattern of iedg_trace_pattern, block
 *         row-major [equation component][unknown component];
 *   R     [n_trace][m] condensed right-hand side.
 * Inputs as in iedg_eval_residual (q required).  The element factors are kept in
 * the handle for iedg_back_substitute. */
int iedg_assemble_condensed(iedg_mesh* mesh, const double* u, const double* q,
                            const double* uhat, const double* u_ref,
                            double* K_bsr, double* R, void* stream);

/* Back-substitution after a trace solve: dZ_e = A_e^-1 (F_e - B_e dU_e) with the
 * factors of the most recent iedg_assemble_condensed on this handle.
 *   duhat [n_trace][m] -> du [n_elem][Np][m], dq [n_elem][Np][m][d].
 * IEDG_ERR_NOT_ASSEMBLED if no assembly has been run. */
int iedg_back_substitute(iedg_mesh* mesh, const double* duhat, double* du, double* dq,
                         void* stream);

/* Per-element status of the last assembly (IEDG_ELEM_*), copied to HOST
 * out[n_elem]; synchronises `stream`.  Returns the number of flagged elements
 * (>= 0) or a negative error code. */
int64_t iedg_element_status(iedg_mesh* mesh, int8_t* out, void* stream);

/* Trace solve K dU = R (Eq. LS) on the GPU: restarted GMRES with iterated classical
 * Gram-Schmidt orthogonalisation and left preconditioning (Sec. 2.2.2), the
 * preconditioner being block Jacobi with the m x m diagonal blocks of K (the one-
 * subdomain, zero-overlap case of the paper's additive Schwarz family).
 *   K  [nnzb][m][m] in the pattern of iedg_trace_pattern, R [n_trace][m]  (device)
 *   dU [n_trace][m] output (device), starts from zero
 *   restart 1..IEDG_MAX_RESTART, max_iter >= 1 (Arnoldi steps in total),
 *   rtol > 0: stop when |M^-1 (R - K dU)| <= rtol |M^-1 R| (the GMRES estimate
 *   during a cycle, recomputed at restarts).
 * Outputs iterations and the final relative preconditioned residual (may be NULL).
 * The Hessenberg matrix, its Givens rotations and the residual estimate are kept and
 * updated on the device; the host reads the estimate once per Arnoldi step (one
 * synchronisation of `stream` per step) to decide when to stop.  Workspace is
 * allocated with the mesh.  IEDG_ERR_INVALID_ARG for a singular diagonal block. */
#define IEDG_MAX_RESTART 40

/* Preconditioner of iedg_trace_solve (default IEDG_PREC_BLOCK_JACOBI).
 *   IEDG_PREC_BILU0: the zero fill-in m x m block incomplete LU of K (BILU(0), Sec.
 *   2.2.2), in multicolour order: trace nodes coloured greedily in index order (each
 *   takes the smallest colour none of its earlier neighbours has, neighbours = nodes
 *   sharing a block of K), then eliminated colour by colour, ties by index.  Nodes of
 *   one colour share no block, so each colour is factored and solved in one launch.
 *   (The paper orders by minimum discarded fill, a sequential CPU ordering.)  The
 *   colouring and per-row orders are built on the first use (host work, one device
 *   buffer of nnzb m^2 doubles for the factors). */
#define IEDG_PREC_BLOCK_JACOBI 0
#define IEDG_PREC_BILU0        1
int iedg_set_trace_precond(iedg_mesh* mesh, int32_t kind);

/* BILU(0) pieces for callers and tests: factors of K in K's layout (blocks of
 * neighbours eliminated before the row hold L, the others U; device F [nnzb][m][m]),
 * the preconditioner solve x = U^-1 L^-1 r with the factors of the most recent
 * iedg_bilu0_factor on this handle (r, x [n_trace][m], device, x may equal r), and the
 * colour of every trace node (HOST int32 [n_trace]).  iedg_bilu0_factor returns
 * IEDG_ERR_INVALID_ARG for an exactly singular pivot block. */
int iedg_bilu0_factor(iedg_mesh* mesh, const double* K, double* F, void* stream);
int iedg_bilu0_apply(iedg_mesh* mesh, const double* F, const double* r, double* x, void* stream);
int iedg_trace_colors(iedg_mesh* mesh, int32_t* colors);
int iedg_trace_solve(iedg_mesh* mesh, const double* K, const double* R, double* dU, int32_t restart,
                     int32_t max_iter, double rtol, int32_t* iterations, double* rel_residual,
                     void* stream);

/* Launch schedule of the batched kernels (no counterpart in the paper; the choices
 * an autotuner sweeps, see paper_1605_01020_gb300/autotune.py).  Results do not
 * depend on it except through floating-point summation order in the LU.
 *   lu_persistent: 1 = the batched LU runs as a persistent grid (resident CTAs per
 *                  SM x SMs) that takes elements from an atomic queue; 0 = one CTA
 *                  per element.
 *   lu_panel:      FP64 LU panel width, 16 or 32 (32 falls back to 16 when the panel
 *                  does not fit in shared memory).
 *   asm_chunk:     assembly column chunk, 8, 16 or 32 (0 = default: 8 for FP64, 16
 *                  for FP32; too large a chunk for shared memory falls back).
 *   lu_tensor:     1 = the Schur complement K = D - W Z of the partial LU on the tensor
 *                  cores (tcgen05, accumulation in tensor memory).  FP64 path: the FP64
 *                  operands are split exactly into integer slices of 7 bits, the slice
 *                  products of equal weight accumulate exactly in FP32 over K chunks of
 *                  64 and are summed in FP64 (results agree with the DFMA form to
 *                  FP64 rounding); the panel factorisation stays on DFMA; persistent
 *                  grid, panel 16; its per-CTA slice buffers (16 (nt + 1) nu floats
 *                  per resident CTA) are allocated by this call when it selects the
 *                  form (IEDG_ERR_OOM if they do not fit), not by the compute calls.  Mixed path: TF32 operands split in high and low
 *                  parts, three products ("3xTF32").  2 (mixed FP32 form only) = every
 *                  trailing update of the FP32 LU on the tensor cores (3xTF32, 128 x 64
 *                  tiles accumulated in TMEM and subtracted from the trailing block by
 *                  reductions in L2).  0 = DFMA / FFMA updates.  Default 0, except 2
 *                  for mixed FP32 handles of meshes with mixed orders.  Handles created with
 *                  IEDG_PRECISION_MIXED_TF32 or _MIXED_BF16 always take the tensor-core
 *                  form in their own operand precision (the schedule never changes
 *                  what is computed, only how).
 *   asm_chunk_by_order[p-1]: meshes with mixed orders: the assembly chunk of the
 *                  elements of order p (8, 16, 32; 0 = asm_chunk), so that each
 *                  order's assembly launch gets its own tuned tile.
 * iedg_set_schedule rejects other values with IEDG_ERR_INVALID_ARG. */
typedef struct {
  int32_t lu_persistent;
  int32_t lu_panel;
  int32_t asm_chunk;
  int32_t lu_tensor;
  int32_t asm_chunk_by_order[4];
} iedg_schedule;
int iedg_get_schedule(const iedg_mesh* mesh, iedg_schedule* out);
int iedg_set_schedule(iedg_mesh* mesh, const iedg_schedule* in);

/* Host-side fault injection for tests of the failure handling (no counterpart in
 * the paper).  Nothing here faults, traps or hangs the GPU: each field makes one
 * kind of element failure happen on purpose so that its status can be checked.
 *   zero_row_elem: element (user id, uniform meshes) whose bordered element matrix
 *                  gets u-row zero_row (0 <= zero_row < m Np) set to zero after
 *                  assembly and before the LU, which makes its element block singular
 *                  (the element must come back IEDG_ELEM_SINGULAR); -1 = none.
 *   refine_iters:  mixed forms: correction steps of the FP64 refinement (0..16, -1 =
 *                  the default 8).  0 leaves the FP32 solve unrefined, so elements
 *                  come back IEDG_ELEM_REFINE.
 *   tc_wait_limit: polls of each tensor-core completion wait (tcgen05 forms) before it
 *                  gives up (0 = the default 2^26; -1 = no poll, every wait gives up at
 *                  once).  A wait that gives up stops its CTA from factoring (after its
 *                  MMAs in flight drain at the default limit and its TMEM is freed);
 *                  that element and every element the CTA still takes from the queue
 *                  come back IEDG_ELEM_TIMEOUT.
 * The settings stay until changed; {-1, 0, -1, 0} restores normal operation.
 * IEDG_ERR_INVALID_ARG for values out of range, IEDG_ERR_UNSUPPORTED for zero_row_elem
 * on meshes with mixed orders. */
typedef struct {
  int64_t zero_row_elem;
  int32_t zero_row;
  int32_t refine_iters;
  int32_t tc_wait_limit;
  int32_t reserved;
} iedg_fault_injection;
int iedg_set_fault_injection(iedg_mesh* mesh, const iedg_fault_injection* f);

/* Residual without any allocation (no counterpart in the paper; a service for
 * callers that cannot allocate device memory when they need a residual, e.g. code
 * whose device memory is owned by a framework pool, real-time loops where the
 * implicit synchronisation of cudaMalloc/cudaFree is not allowed, or plug-ins that
 * are given buffers but no allocation rights).  Same result as iedg_eval_residual
 * with a given q: r_u [n_elem][Np][m] (may be NULL) and r_fl [n_trace][m].  q is
 * required (no lifting), r_q is not produced.
 * Scratch: the per-element trace residuals go to one file-scope device array of
 * IEDG_STATIC_SCRATCH_DOUBLES doubles (16 MiB) that every GPU loading the library
 * holds until the process exits; meshes with n_elem * Nb * m above that are
 * rejected with IEDG_ERR_INVALID_ARG.  The array is shared by all calls and keeps
 * the last call's contents (every entry read is written first in the same call):
 * calls that overlap on the GPU (other streams, other handles) race on it and must
 * be serialised by the caller.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  No cudaMalloc, cudaFree or allocating library
 * routine is called.  Kernel launches of this entry point are not traced. */
#define IEDG_STATIC_SCRATCH_DOUBLES (1u << 21)
int iedg_eval_residual_static(iedg_mesh* mesh, const double* u, const double* uhat,
                              const double* q, const double* u_ref, double* r_u,
                              double* r_fl, void* stream);

/* Tracing (no counterpart in the paper; it times the library's own kernels).
 * Every kernel launch is counted per kernel name.  While profiling is enabled,
 * each launch is also bracketed by CUDA events recorded on the launching stream,
 * so the summed device time per kernel is available.  iedg_profile_read fills up
 * to max_kernels entries: names[i] (NUL-terminated, 32 bytes each), launches[i],
 * ms[i] (0 unless profiling was enabled), and sets *n_kernels; it synchronises
 * the recorded events.  iedg_profile_reset clears counts, times and events. */
int iedg_profile_enable(iedg_mesh* mesh, int32_t enable);
int iedg_profile_read(iedg_mesh* mesh, int32_t max_kernels, char* names, int64_t* launches,
                      double* ms, int32_t* n_kernels);
int iedg_profile_reset(iedg_mesh* mesh);

#ifdef __cplusplus
}
#endif
#endif /* IEDG_H */
