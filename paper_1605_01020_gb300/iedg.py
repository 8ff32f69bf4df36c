"""Thin ctypes binding of the C ABI in include/iedg.h (argument marshalling only).

Every step of the computation runs in libiedg.so's CUDA kernels; this module only
checks shapes/dtypes, passes device pointers of torch tensors and the current CUDA
stream, and turns error codes into exceptions.  There is no CPU fallback: if the
shared library is missing or no GPU is present, calls raise.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libiedg.so")

OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "MESH", -5: "NOT_ASSEMBLED", -6: "UNSUPPORTED"}
EXPORTS = ("iedg_create_mesh", "iedg_destroy_mesh", "iedg_last_error", "iedg_mesh_info",
           "iedg_trace_pattern", "iedg_eval_residual", "iedg_assemble_condensed",
           "iedg_back_substitute", "iedg_element_status", "iedg_profile_enable",
           "iedg_profile_read", "iedg_profile_reset", "iedg_eval_residual_static", "iedg_get_schedule",
           "iedg_set_schedule", "iedg_trace_solve", "iedg_create_mesh_mixed", "iedg_element_sizes",
           "iedg_set_trace_precond", "iedg_bilu0_factor", "iedg_bilu0_apply", "iedg_trace_colors",
           "iedg_create_mesh_bc", "iedg_set_fault_injection")
PREC_BLOCK_JACOBI, PREC_BILU0 = 0, 1
# element-matrix precision of a handle (IEDG_PRECISION_*)
PRECISION_FP64, PRECISION_MIXED, PRECISION_MIXED_TF32, PRECISION_MIXED_BF16 = 0, 1, 2, 3
# per-element status codes (IEDG_ELEM_*)
ELEM_OK, ELEM_REFINE, ELEM_SINGULAR, ELEM_NONFINITE, ELEM_TIMEOUT, ELEM_FALLBACK = 0, 1, 2, 3, 4, 5


class IedgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"iedg error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class MeshDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("order", ctypes.c_int32), ("quad_extra", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("n_elem", ctypes.c_int64), ("n_trace", ctypes.c_int64),
                ("node_xyz", ctypes.c_void_p), ("elem_trace", ctypes.c_void_p),
                ("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("Re", ctypes.c_double),
                ("Minf", ctypes.c_double), ("alpha", ctypes.c_double), ("stab", ctypes.c_int32),
                ("flags", ctypes.c_int32)]
FLAG_MASS_SCALING = 1


class Schedule(ctypes.Structure):
    _fields_ = [("lu_persistent", ctypes.c_int32), ("lu_panel", ctypes.c_int32), ("asm_chunk", ctypes.c_int32),
                ("lu_tensor", ctypes.c_int32), ("asm_chunk_by_order", ctypes.c_int32 * 4)]


class FaultInjection(ctypes.Structure):
    _fields_ = [("zero_row_elem", ctypes.c_int64), ("zero_row", ctypes.c_int32), ("refine_iters", ctypes.c_int32),
                ("tc_wait_limit", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None


def load():
    """Load libiedg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built: run __graft_entry__.build() or "
                          f"python -m paper_1605_01020_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.iedg_create_mesh.argtypes = [ctypes.POINTER(MeshDesc), vp, ctypes.POINTER(vp)]
    lib.iedg_create_mesh.restype = ctypes.c_int
    lib.iedg_create_mesh_mixed.argtypes = [ctypes.POINTER(MeshDesc), vp, vp, vp, ctypes.POINTER(vp)]
    lib.iedg_create_mesh_mixed.restype = ctypes.c_int
    lib.iedg_create_mesh_bc.argtypes = [ctypes.POINTER(MeshDesc), vp, vp, vp, vp, vp, ctypes.POINTER(vp)]
    lib.iedg_create_mesh_bc.restype = ctypes.c_int
    lib.iedg_element_sizes.argtypes = [vp, vp, vp]
    lib.iedg_element_sizes.restype = ctypes.c_int
    lib.iedg_destroy_mesh.argtypes = [vp]
    lib.iedg_destroy_mesh.restype = ctypes.c_int
    lib.iedg_last_error.argtypes = [vp]
    lib.iedg_last_error.restype = ctypes.c_char_p
    lib.iedg_mesh_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64),
                                   ctypes.POINTER(i64)]
    lib.iedg_mesh_info.restype = ctypes.c_int
    lib.iedg_trace_pattern.argtypes = [vp, vp, vp, vp]
    lib.iedg_trace_pattern.restype = ctypes.c_int
    lib.iedg_eval_residual.argtypes = [vp] * 10
    lib.iedg_eval_residual.restype = ctypes.c_int
    lib.iedg_assemble_condensed.argtypes = [vp] * 8
    lib.iedg_assemble_condensed.restype = ctypes.c_int
    lib.iedg_back_substitute.argtypes = [vp] * 5
    lib.iedg_back_substitute.restype = ctypes.c_int
    lib.iedg_element_status.argtypes = [vp, vp, vp]
    lib.iedg_element_status.restype = ctypes.c_int64
    lib.iedg_eval_residual_static.argtypes = [vp] * 8
    lib.iedg_eval_residual_static.restype = ctypes.c_int
    lib.iedg_trace_solve.argtypes = [vp, vp, vp, vp, i32, i32, ctypes.c_double, ctypes.POINTER(i32),
                                     ctypes.POINTER(ctypes.c_double), vp]
    lib.iedg_trace_solve.restype = ctypes.c_int
    lib.iedg_set_trace_precond.argtypes = [vp, i32]
    lib.iedg_set_trace_precond.restype = ctypes.c_int
    lib.iedg_bilu0_factor.argtypes = [vp, vp, vp, vp]
    lib.iedg_bilu0_factor.restype = ctypes.c_int
    lib.iedg_bilu0_apply.argtypes = [vp, vp, vp, vp, vp]
    lib.iedg_bilu0_apply.restype = ctypes.c_int
    lib.iedg_trace_colors.argtypes = [vp, vp]
    lib.iedg_trace_colors.restype = ctypes.c_int
    lib.iedg_get_schedule.argtypes = [vp, ctypes.POINTER(Schedule)]
    lib.iedg_get_schedule.restype = ctypes.c_int
    lib.iedg_set_schedule.argtypes = [vp, ctypes.POINTER(Schedule)]
    lib.iedg_set_schedule.restype = ctypes.c_int
    lib.iedg_set_fault_injection.argtypes = [vp, ctypes.POINTER(FaultInjection)]
    lib.iedg_set_fault_injection.restype = ctypes.c_int
    lib.iedg_profile_enable.argtypes = [vp, i32]
    lib.iedg_profile_enable.restype = ctypes.c_int
    lib.iedg_profile_read.argtypes = [vp, i32, vp, vp, vp, ctypes.POINTER(i32)]
    lib.iedg_profile_read.restype = ctypes.c_int
    lib.iedg_profile_reset.argtypes = [vp]
    lib.iedg_profile_reset.restype = ctypes.c_int
    _lib = lib
    return lib


def _torch():
    import torch
    return torch


def _ptr(t, shape=None, dtype=None, name="tensor"):
    if t is None:
        return None
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr()


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Mesh:
    """Handle around iedg_create_mesh / iedg_destroy_mesh with the compute calls."""

    def __init__(self, node_xyz, elem_trace, n_trace, order, gamma=1.4, Pr=0.72, Re=1e3, Minf=0.2,
                 alpha=0.0, quad_extra=2, precision=0, stream=None, stab=0, flags=0):
        lib = load()
        X = np.ascontiguousarray(node_xyz, dtype=np.float64)
        ET = np.ascontiguousarray(elem_trace, dtype=np.int64)
        self.E, self.Np_in, self.d = X.shape
        self.m = self.d + 2
        self.T = int(n_trace)
        self.order = int(order)
        self.alpha = float(alpha)
        desc = MeshDesc(self.d, self.order, quad_extra, precision, self.E, self.T,
                        X.ctypes.data, ET.ctypes.data, gamma, Pr, Re, Minf, alpha, int(stab), int(flags))
        h = ctypes.c_void_p()
        rc = lib.iedg_create_mesh(ctypes.byref(desc), ctypes.c_void_p(_stream(stream)), ctypes.byref(h))
        if rc != OK:
            raise IedgError(rc, lib.iedg_last_error(None).decode())
        self._h = h
        self._info()
        if self.Np != self.Np_in or ET.shape != (self.E, self.Nb):
            raise ValueError("node_xyz / elem_trace shapes do not match the order")
        self._ushape = (self.E, self.Np, self.m)
        self._qshape = (self.E, self.Np, self.m, self.d)

    def _info(self):
        np_, nb, nnzb, ws = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        self._check(load().iedg_mesh_info(self._h, ctypes.byref(np_), ctypes.byref(nb), ctypes.byref(nnzb),
                                          ctypes.byref(ws)))
        self.Np, self.Nb, self.nnzb, self.workspace_bytes = np_.value, nb.value, nnzb.value, ws.value

    def element_sizes(self):
        """(Np_e, nb_e) per element, numpy int32 arrays."""
        npe = np.zeros(self.E, dtype=np.int32)
        nbe = np.zeros(self.E, dtype=np.int32)
        self._check(load().iedg_element_sizes(self._h, npe.ctypes.data, nbe.ctypes.data))
        return npe, nbe

    def _check(self, rc):
        if rc != OK:
            raise IedgError(rc, load().iedg_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().iedg_destroy_mesh(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ helpers
    def _empty(self, *shape, dtype=None):
        torch = _torch()
        return torch.empty(*shape, dtype=dtype or torch.float64, device="cuda")

    def trace_pattern(self, stream=None):
        torch = _torch()
        row_ptr = self._empty(self.T + 1, dtype=torch.int64)
        col = self._empty(self.nnzb, dtype=torch.int32)
        self._check(load().iedg_trace_pattern(self._h, row_ptr.data_ptr(), col.data_ptr(), _stream(stream)))
        return row_ptr, col

    def eval_residual(self, u, uhat, q=None, u_ref=None, q_out=None, r_q=None, r_u=None, r_fl=None,
                      stream=None, want=("r_q", "r_u", "r_fl")):
        torch = _torch()
        m, T, us, qs = self.m, self.T, self._ushape, self._qshape
        f64 = torch.float64
        if q is None and q_out is None:
            q_out = self._empty(*qs)
        if r_q is None and "r_q" in want:
            r_q = self._empty(*qs)
        if r_u is None and "r_u" in want:
            r_u = self._empty(*us)
        if r_fl is None and "r_fl" in want:
            r_fl = self._empty(T, m)
        self._check(load().iedg_eval_residual(
            self._h, _ptr(u, us, f64, "u"), _ptr(uhat, (T, m), f64, "uhat"),
            _ptr(q, qs, f64, "q"), _ptr(u_ref, us, f64, "u_ref"),
            _ptr(q_out, qs, f64, "q_out"), _ptr(r_q, qs, f64, "r_q"),
            _ptr(r_u, us, f64, "r_u"), _ptr(r_fl, (T, m), f64, "r_fl"), _stream(stream)))
        return dict(q=q_out if q is None else q, r_q=r_q, r_u=r_u, r_fl=r_fl)

    def assemble_condensed(self, u, q, uhat, u_ref=None, K=None, R=None, stream=None):
        torch = _torch()
        m, T, us, qs = self.m, self.T, self._ushape, self._qshape
        f64 = torch.float64
        K = self._empty(self.nnzb, m, m) if K is None else K
        R = self._empty(T, m) if R is None else R
        self._check(load().iedg_assemble_condensed(
            self._h, _ptr(u, us, f64, "u"), _ptr(q, qs, f64, "q"),
            _ptr(uhat, (T, m), f64, "uhat"), _ptr(u_ref, us, f64, "u_ref"),
            _ptr(K, (self.nnzb, m, m), f64, "K"), _ptr(R, (T, m), f64, "R"), _stream(stream)))
        return K, R

    def back_substitute(self, duhat, du=None, dq=None, stream=None):
        torch = _torch()
        m, T, us, qs = self.m, self.T, self._ushape, self._qshape
        f64 = torch.float64
        du = self._empty(*us) if du is None else du
        dq = self._empty(*qs) if dq is None else dq
        self._check(load().iedg_back_substitute(
            self._h, _ptr(duhat, (T, m), f64, "duhat"), _ptr(du, us, f64, "du"),
            _ptr(dq, qs, f64, "dq"), _stream(stream)))
        return du, dq

    def element_status(self, stream=None):
        out = np.zeros(self.E, dtype=np.int8)
        rc = load().iedg_element_status(self._h, out.ctypes.data, _stream(stream))
        if rc < 0:
            self._check(int(rc))
        return out


    def trace_solve(self, K, R, dU=None, restart=30, max_iter=400, rtol=1e-10, stream=None):
        """GMRES / block-Jacobi solve of K dU = R; returns (dU, iterations, rel_residual)."""
        torch = _torch()
        m, T = self.m, self.T
        f64 = torch.float64
        dU = self._empty(T, m) if dU is None else dU
        it, rr = ctypes.c_int32(), ctypes.c_double()
        self._check(load().iedg_trace_solve(
            self._h, _ptr(K, (self.nnzb, m, m), f64, "K"), _ptr(R, (T, m), f64, "R"), _ptr(dU, (T, m), f64, "dU"),
            restart, max_iter, rtol, ctypes.byref(it), ctypes.byref(rr), _stream(stream)))
        return dU, it.value, rr.value

    def set_trace_precond(self, kind):
        """PREC_BLOCK_JACOBI (default) or PREC_BILU0 for trace_solve."""
        self._check(load().iedg_set_trace_precond(self._h, int(kind)))

    def bilu0_factor(self, K, F=None, stream=None):
        torch = _torch()
        m = self.m
        F = self._empty(self.nnzb, m, m) if F is None else F
        self._check(load().iedg_bilu0_factor(self._h, _ptr(K, (self.nnzb, m, m), torch.float64, "K"),
                                             _ptr(F, (self.nnzb, m, m), torch.float64, "F"), _stream(stream)))
        return F

    def bilu0_apply(self, F, r, x=None, stream=None):
        torch = _torch()
        m, T = self.m, self.T
        x = self._empty(T, m) if x is None else x
        self._check(load().iedg_bilu0_apply(self._h, _ptr(F, (self.nnzb, m, m), torch.float64, "F"),
                                            _ptr(r, (T, m), torch.float64, "r"), _ptr(x, (T, m), torch.float64, "x"),
                                            _stream(stream)))
        return x

    def trace_colors(self):
        out = np.zeros(self.T, dtype=np.int32)
        self._check(load().iedg_trace_colors(self._h, out.ctypes.data))
        return out

    # ------------------------------------------------------------------ schedule
    def get_schedule(self):
        sc = Schedule()
        self._check(load().iedg_get_schedule(self._h, ctypes.byref(sc)))
        out = {"lu_persistent": sc.lu_persistent, "lu_panel": sc.lu_panel, "asm_chunk": sc.asm_chunk,
               "lu_tensor": sc.lu_tensor}
        if any(sc.asm_chunk_by_order):
            out["asm_chunk_by_order"] = list(sc.asm_chunk_by_order)
        return out

    def set_schedule(self, **kw):
        cur = self.get_schedule()
        cur.update(kw)
        by = (ctypes.c_int32 * 4)(*cur.get("asm_chunk_by_order", [0, 0, 0, 0]))
        sc = Schedule(cur["lu_persistent"], cur["lu_panel"], cur["asm_chunk"], cur["lu_tensor"], by)
        self._check(load().iedg_set_schedule(self._h, ctypes.byref(sc)))

    def set_fault_injection(self, zero_row_elem=-1, zero_row=0, refine_iters=-1, tc_wait_limit=0):
        """Host-side fault injection for tests (iedg_set_fault_injection); the defaults
        restore normal operation."""
        f = FaultInjection(int(zero_row_elem), int(zero_row), int(refine_iters), int(tc_wait_limit), 0)
        self._check(load().iedg_set_fault_injection(self._h, ctypes.byref(f)))

    # ------------------------------------------------------------------ tracing
    def profile_enable(self, enable=True):
        self._check(load().iedg_profile_enable(self._h, 1 if enable else 0))

    def profile_reset(self):
        self._check(load().iedg_profile_reset(self._h))

    def profile_read(self):
        """{kernel name: (launches, summed device ms)}; synchronises the events."""
        cap = 64
        names = ctypes.create_string_buffer(32 * cap)
        launches = np.zeros(cap, dtype=np.int64)
        ms = np.zeros(cap, dtype=np.float64)
        n = ctypes.c_int32()
        self._check(load().iedg_profile_read(self._h, cap, names, launches.ctypes.data, ms.ctypes.data,
                                             ctypes.byref(n)))
        out = {}
        for i in range(min(n.value, cap)):
            nm = names.raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
            out[nm] = (int(launches[i]), float(ms[i]))
        return out


def _slot_count(d, p, fdeg, _cache={}):
    """Trace slots of an element of order p with face degrees fdeg (see
    iedg_create_mesh_mixed): boundary nodes on faces of degree 0, plus (q+1)^(d-1)
    private nodes per face of degree q > 0."""
    key = (d, p, fdeg)
    if key not in _cache:
        idx = np.stack(np.meshgrid(*[np.arange(p + 1)] * d, indexing="ij"), -1).reshape(-1, d)
        on = np.zeros(len(idx), dtype=bool)
        for f, q in enumerate(fdeg):
            if q == 0:
                on |= idx[:, f // 2] == (p if f % 2 else 0)
        _cache[key] = int(on.sum()) + sum((q + 1) ** (d - 1) for q in fdeg if q > 0)
    return _cache[key]


class MixedOrderMesh(Mesh):
    """Handle around iedg_create_mesh_mixed: elements of different orders sharing one
    trace space.  Element-indexed arrays are ragged, elements in the given order, each
    with its own number of nodes: u [sum Np_e, m], q [sum Np_e, m, d]."""

    def __init__(self, node_xyz, elem_trace, n_trace, orders, face_degree, gamma=1.4, Pr=0.72, Re=1e3,
                 Minf=0.2, alpha=0.0, quad_extra=2, precision=0, stream=None, stab=0, face_kind=None,
                 u_far=None):
        lib = load()
        X = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64) for x in node_xyz]))
        ET = np.ascontiguousarray(np.concatenate([np.asarray(t, dtype=np.int64) for t in elem_trace]))
        ORD = np.ascontiguousarray(orders, dtype=np.int32)
        FD = np.ascontiguousarray(face_degree, dtype=np.int32)
        self.E = len(ORD)
        self.d = X.shape[1]
        self.m = self.d + 2
        self.T = int(n_trace)
        self.order = 0
        self.alpha = float(alpha)
        if FD.shape != (self.E, 2 * self.d):
            raise ValueError("face_degree must be [n_elem, 2 d]")
        # the library reads the ragged arrays with the sizes the orders and face degrees
        # imply: check them here, before any pointer is passed
        for e in range(self.E):
            if len(node_xyz[e]) != (int(ORD[e]) + 1) ** self.d or \
                    len(elem_trace[e]) != _slot_count(self.d, int(ORD[e]), tuple(FD[e].tolist())):
                raise ValueError(f"element {e}: node_xyz / elem_trace sizes do not match its order and face degrees")
        desc = MeshDesc(self.d, 0, quad_extra, precision, self.E, self.T,
                        X.ctypes.data, ET.ctypes.data, gamma, Pr, Re, Minf, alpha, int(stab), 0)
        h = ctypes.c_void_p()
        FK = None if face_kind is None else np.ascontiguousarray(face_kind, dtype=np.int32)
        if FK is not None and FK.shape != FD.shape:
            raise ValueError("face_kind must be [n_elem, 2 d]")
        UF = None if u_far is None else np.ascontiguousarray(u_far, dtype=np.float64)
        if UF is not None and UF.shape != (self.m,):
            raise ValueError("u_far must have m entries")
        rc = lib.iedg_create_mesh_bc(ctypes.byref(desc), ORD.ctypes.data, FD.ctypes.data,
                                     None if FK is None else FK.ctypes.data,
                                     None if UF is None else UF.ctypes.data,
                                     ctypes.c_void_p(_stream(stream)), ctypes.byref(h))
        if rc != OK:
            raise IedgError(rc, lib.iedg_last_error(None).decode())
        self._h = h
        self._info()
        npe, nbe = self.element_sizes()
        self.node_off = np.concatenate([[0], np.cumsum(npe.astype(np.int64))])
        self.n_nodes = int(self.node_off[-1])
        if self.n_nodes != X.shape[0] or int(nbe.sum()) != ET.shape[0]:
            raise ValueError("node_xyz / elem_trace sizes do not match the orders and face degrees")
        self._ushape = (self.n_nodes, self.m)
        self._qshape = (self.n_nodes, self.m, self.d)
        counts = np.bincount(ORD, minlength=5)
        self.orders_present = [p for p, c in enumerate(counts) if c]
        self.orders_key = "|orders" + ",".join(f"{p}:{c}" for p, c in enumerate(counts) if c) + f"|E{self.E}"


def mesh_from_workload(wl, precision=0, stream=None, quad_extra=2, flags=0):
    """Convenience: a Mesh for a workloads.Workload."""
    p = wl.params
    return Mesh(wl.mesh.node_xyz, wl.mesh.elem_trace, wl.mesh.n_trace, wl.mesh.p, gamma=p["gamma"],
                Pr=p["Pr"], Re=p["Re"], Minf=p["Minf"], alpha=p["alpha"], precision=precision, stream=stream,
                stab=p.get("stab", 0), quad_extra=quad_extra, flags=flags)
