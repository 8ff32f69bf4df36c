"""Launch-schedule autotuner for the batched element kernels.

For one mesh (fixed dimension, order, quadrature and precision) it times
iedg_assemble_condensed under every candidate iedg_schedule (persistent or
one-CTA-per-element LU, FP64 LU panel width, assembly column chunk) with CUDA
events, keeps the fastest, and caches the choice in a JSON file keyed by the GPU
name and the mesh class, so later runs on the same kind of GPU skip the sweep.
Results do not depend on the schedule (beyond summation order in the LU).
"""
import itertools
import json
import os

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "iedg", "schedules.json")


def mesh_key(mesh, precision, gpu_name):
    extra = getattr(mesh, "orders_key", "")
    return f"{gpu_name}|d{mesh.d}|p{mesh.order}|Np{mesh.Np}|prec{precision}{extra}"


def candidates(precision, order):
    """Candidate schedules: persistent LU on/off x FP64 panel 16/32 x assembly chunk,
    and the tensor-core forms (the FP64 Schur complement by exact operand splitting;
    on the mixed path the FP32 LU with every trailing update in 3xTF32, or only its
    deferred Schur complement; handles with TF32 or BF16 Schur operands always take
    the tensor-core form).
    order 0 (mixed orders): the FP64 panel stays 16 (the largest elements' panel of
    32 does not fit in shared memory)."""
    panels = [16, 32] if (precision == 0 and 1 <= order <= 3) else [16]
    chunks = [8, 16] if precision == 0 else [16, 32]
    if precision == 0:
        # DFMA forms, then the tensor-core Schur form (persistent, panel 16 only)
        out = [dict(lu_persistent=a, lu_panel=b, asm_chunk=c, lu_tensor=0)
               for a, b, c in itertools.product([1, 0], panels, chunks)]
        return out + [dict(lu_persistent=1, lu_panel=16, asm_chunk=c, lu_tensor=1) for c in chunks]
    # TF32 / BF16 Schur operands: the tensor-core form is what the precision means.
    # FP32 form: every trailing update on the tensor cores (2), the deferred Schur
    # complement on the tensor cores (1), or FFMA updates (0)
    tensor = [2, 1, 0] if precision == 1 else [1]
    return [dict(lu_persistent=a, lu_panel=b, asm_chunk=c, lu_tensor=t)
            for a, b, c, t in itertools.product([1, 0], panels, chunks, tensor)]


def time_assemble(mesh, u, q, uh, K, R, reps, warm=True):
    import torch
    if warm:
        mesh.assemble_condensed(u, q, uh, K=K, R=R)      # warm-up (kernel attributes, caches)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        mesh.assemble_condensed(u, q, uh, K=K, R=R)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(mesh, u, q, uh, precision, reps=2, cache_path=DEFAULT_CACHE, use_cache=True):
    """Pick the fastest schedule for `mesh` on the current GPU, apply it, and return
    (schedule, {candidate: ms}).  `u, q, uh` are device inputs of the mesh."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = mesh_key(mesh, precision, gpu)
    cache = {}
    if use_cache and cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        mesh.set_schedule(**cache[key]["schedule"])
        return cache[key]["schedule"], cache[key].get("timings", {})
    K = torch.empty(mesh.nnzb, mesh.m, mesh.m, dtype=torch.float64, device=u.device)
    R = torch.empty(mesh.T, mesh.m, dtype=torch.float64, device=u.device)
    timings = {}
    best, best_ms = None, float("inf")
    orders = getattr(mesh, "orders_present", None)
    cands = candidates(precision, mesh.order)
    if orders:
        # mixed orders: LU variants first (every order at the default chunk), then each
        # order's assembly chunk on its own (the orders' assembly launches are separate
        # and run one after another, so their times add up)
        cands = [c for c in cands if c["asm_chunk"] == cands[0]["asm_chunk"]]
    first = True
    for cand in cands:
        mesh.set_schedule(**cand)
        ms = time_assemble(mesh, u, q, uh, K, R, reps, warm=first)
        first = False
        timings[json.dumps(cand, sort_keys=True)] = ms
        if ms < best_ms:
            best, best_ms = cand, ms
    if orders:
        chunks = [8, 16] if precision == 0 else [16, 32]
        by = [0, 0, 0, 0]
        for p in orders:
            best_c, best_c_ms = None, float("inf")
            for c in chunks:
                trial = list(by)
                trial[p - 1] = c
                cand = dict(best, asm_chunk_by_order=trial)
                mesh.set_schedule(**cand)
                ms = time_assemble(mesh, u, q, uh, K, R, reps, warm=False)
                timings[json.dumps(cand, sort_keys=True)] = ms
                if ms < best_c_ms:
                    best_c, best_c_ms = c, ms
            by[p - 1] = best_c
        best = dict(best, asm_chunk_by_order=by)
    mesh.set_schedule(**best)
    if cache_path:
        cache[key] = {"schedule": best, "timings": timings}
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
        except OSError:
            pass
    return best, timings
