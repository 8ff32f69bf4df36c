#!/usr/bin/env python
"""Benchmark of the IEDG element-local Newton step on GB300.

One step = one pass of the whole element-local hot path over the 3D p=3 16^3
periodic workload (4096 curved-capable hexes, FP64):
    iedg_eval_residual      (q lifted from R_q = 0, R_q, R_u, R_FL)
    iedg_assemble_condensed (point Jacobians, element blocks with q eliminated,
                             batched partial LU / Schur complement, BSR scatter)
    iedg_back_substitute    (element updates from a trace increment)
Metric: condensed elements per second.  Inputs are resident in HBM when the timed
region starts; `e2e` repeats the measurement through the same public API with the
inputs copied from pinned host memory and the results (K, R, du, dq) copied back
inside the timed region.

Multi-GPU: every rank condenses its own mesh of the same size (the element-local
path has no exchange step), so scaling is weak and value = all ranks' elements /
max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "elements/s condensed (3D NS, p=3) FP64 vs mixed+refine; % tensor roofline"
DFMA_PER_CLK_PER_SM = 2          # GB300: 1.25 TFLOP/s FP64 at 2070 MHz over 152 SMs
FFMA_PER_CLK_PER_SM = 128        # FP32 FMA lanes per SM per clock


def a6_flops(nu, nt):
    """Algorithmic flops of the partial LU / Schur complement of one bordered element
    matrix with nu pivot columns, nt trace columns and one right-hand side."""
    n = nu + nt
    return sum((n - k - 1) + 2 * (n - k - 1) * (n - k) + 2 * (n - k - 1) for k in range(nu))


def a4a5_flops(d, p, nq1):
    """Algorithmic flops of element-block assembly (A_uu, A_uq volume and face terms)
    plus the q-elimination, the fixed dense-count formulas for one element."""
    m = d + 2
    Np, Nq, Nb = (p + 1) ** d, nq1 ** d, (p + 1) ** d - (p - 1) ** d
    Nfp, Nfq = (p + 1) ** (d - 1), nq1 ** (d - 1)
    a4v = 2 * m * m * d * Np * Np * Nq * (1 + d)
    a4f = 2 * d * (4 * m * m + 2 * m * m * d) * 2 * Nfp * Nfp * Nfq
    a5 = 2 * m * m * d * (Np ** 3 + 2 * Np * Np * Nb + Np * Nb * Nb)
    return a4v + a4f + a5


def assemble_actual_flops(d, p, nq1):
    """Flops the sum-factorised 3D assembly kernel performs per element: right-operand
    build, three 1D contraction stages over the volume points, two 1D stages per face,
    for every (equation, unknown) component pair; pairs whose viscous Jacobian is zero
    skip the lifted-gradient terms."""
    m = d + 2
    np1 = p + 1
    Np, Nq, Nb = np1 ** d, nq1 ** d, np1 ** d - (p - 1) ** d
    Nfq, Nfn = nq1 ** (d - 1), np1 ** (d - 1)
    TS, VS = nq1 * nq1 * np1, nq1 * np1 * np1
    ncol = Np + Nb
    fma = 0
    for i in range(m):
        for k in range(m):
            cq = not (i == 0 or (i <= d and k == m - 1))
            build = Nq * (Np * 3 * (1 + (d if cq else 0)) + (Nb * 3 * d if cq else 0))
            stages = ncol * (3 * TS * nq1 + VS * 3 * nq1 + Np * 2 * nq1)
            face = 2 * d * (Nfq * (Np * (1 + (d if cq else 0)) + Nb * (1 + (d if cq else 0)))
                            + ncol * (nq1 * np1 * nq1 + Nfn * nq1))
            fma += build + stages + face
    return 2 * fma


def traffic_record(kernel, precision, dims):
    """DRAM bytes per element of `kernel` from the committed ncu record, or None when
    there is none for these element sizes or the kernel's source has changed since the
    counters were taken (the record keeps the source file's SHA-256)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    for ln in open(path):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        rec = json.loads(ln)
        if rec["kernel"] != kernel or rec["precision"] != precision or list(rec["dims"]) != list(dims):
            continue
        src = os.path.join(ROOT, rec["source"])
        if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["sha256"]:
            return None
        return float(rec["bytes_per_element"])
    return None


def workload_name(wl):
    return f"{wl.name} ({wl.mesh.n_elem} elements), FP64: residual + condensed trace Jacobian + back-substitution"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def unit_peaks():
    """Measured peak rates of the arithmetic units (TFLOP/s) from the committed probe
    record profiles/peaks_gb300.txt (its last JSON line), or {} when absent."""
    path = os.path.join(ROOT, "profiles", "peaks_gb300.txt")
    if not os.path.exists(path):
        return {}
    lines = [ln for ln in open(path) if ln.strip().startswith("{")]
    return json.loads(lines[-1]) if lines else {}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------------ oracle baseline
def _oracle_elements(args):
    """Worker of the oracle baseline: residual, q-eliminated condensation and
    back-substitution of each listed element, one element at a time (the oracle as
    it stands).  Returns the count done."""
    wl, els = args
    from oracle import geometry, physics, refelem
    from oracle import iedg as oiedg
    st = wl.state
    ref = refelem.RefElement(wl.mesh.d, wl.mesh.p)
    prm = physics.Params(**{k: wl.params[k] for k in ("gamma", "Pr", "Re", "Minf", "alpha")})
    for e in els:
        one = np.array([e])
        geo = geometry.Geometry(ref, wl.mesh.node_xyz[one])
        pb = oiedg.Problem(ref, geo, wl.mesh.elem_trace[one], wl.mesh.n_trace, prm)
        q = pb.solve_q(st.u[one], st.uhat)
        pb.residual(st.u[one], q, st.uhat)
        pb.condense_qelim(0, st.u[one], q, st.uhat)
        pb.back_substitute_qelim(0, st.u[one], q, st.uhat, st.duhat)
    return len(els)


def _worker_init():
    os.environ["OMP_NUM_THREADS"] = "1"
    try:
        from threadpoolctl import threadpool_limits
        threadpool_limits(1)
    except Exception:
        pass


class OraclePool:
    """The CPU oracle on every host core: a process pool (spawn start, so it may be
    created after CUDA work in the parent) with one single-threaded worker per core,
    each taking its own elements."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        self.procs = procs or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_worker_init)

    def run(self, wl, elems):
        """Elements `elems` spread over the workers; returns wall seconds."""
        chunks = [elems[w::self.procs] for w in range(self.procs)]
        chunks = [c for c in chunks if len(c)]
        t0 = time.perf_counter()
        done = sum(self.pool.map(_oracle_elements, [(wl, c) for c in chunks]))
        assert done == len(elems)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_sample(wl, budget_s, procs=None):
    """Time the CPU oracle (as it stands) on a bounded sample of the workload's
    elements spread over all host cores.  The sample size is set from one element
    timed in this process so that the timed run takes about budget_s.
    Returns (elements, seconds, processes)."""
    _worker_init()
    t0 = time.perf_counter()
    _oracle_elements((wl, [0]))
    t1 = time.perf_counter() - t0
    pool = OraclePool(procs)
    try:
        pool.run(wl, list(range(pool.procs)))                       # imports and first calls in every worker
        n = int(min(wl.mesh.n_elem, max(pool.procs, pool.procs * max(1, int(budget_s / max(t1, 1e-3))))))
        secs = pool.run(wl, list(range(n)))
    finally:
        pool.close()
    return n, secs, pool.procs


def run_reference(args, wl, rank):
    """--impl reference: the CPU oracle on the host cores (one single-threaded worker
    process per core), each step a bounded sample of the same workload."""
    if rank != 0:
        return
    pool = OraclePool()
    per_step = max(pool.procs, args.ref_elems * pool.procs)
    try:
        pool.run(wl, list(range(pool.procs)))                       # imports and first calls
        for _ in range(args.warmup):
            pool.run(wl, list(range(min(per_step, wl.mesh.n_elem))))
        el, tot = 0.0, 0
        for _ in range(args.steps):
            els = list(range(min(per_step, wl.mesh.n_elem)))
            el += pool.run(wl, els)
            tot += len(els)
    finally:
        pool.close()
    value = tot / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(wl), "elements": wl.mesh.n_elem,
                                            "order": wl.mesh.p},
            "cpu_baseline": {"value": value, "unit": "elements/s", "cores": pool.procs, "kind": "oracle",
                             "sample": f"{min(per_step, wl.mesh.n_elem)} elements per step (of {wl.mesh.n_elem}), "
                                       f"numpy/scipy FP64 oracle, q-eliminated form, one single-threaded "
                                       f"process per host core"},
            "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args, wl, rank, world, local_rank):
    import torch
    from paper_1605_01020_gb300 import build, iedg

    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    mesh = iedg.mesh_from_workload(wl)
    E, Np, m, d, T = mesh.E, mesh.Np, mesh.m, mesh.d, mesh.T
    st = wl.state
    f64 = torch.float64
    u = torch.as_tensor(st.u, dtype=f64, device=dev)
    uh = torch.as_tensor(st.uhat, dtype=f64, device=dev)
    duh = torch.as_tensor(st.duhat, dtype=f64, device=dev)
    schedule, timings64 = None, {}
    if not args.no_autotune:
        from paper_1605_01020_gb300 import autotune
        qt = torch.as_tensor(st.q, dtype=f64, device=dev)
        schedule, timings64 = autotune.autotune(mesh, u, qt, uh, 0, reps=1)
        del qt
    q = torch.empty(E, Np, m, d, dtype=f64, device=dev)
    rq = torch.empty_like(q)
    ru = torch.empty(E, Np, m, dtype=f64, device=dev)
    rfl = torch.empty(T, m, dtype=f64, device=dev)
    K = torch.empty(mesh.nnzb, m, m, dtype=f64, device=dev)
    R = torch.empty(T, m, dtype=f64, device=dev)
    du = torch.empty(E, Np, m, dtype=f64, device=dev)
    dq = torch.empty_like(q)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    def step(u_, uh_, duh_, outs=None):
        K_, R_, du_, dq_ = outs if outs is not None else (K, R, du, dq)
        mesh.eval_residual(u_, uh_, q=None, q_out=q, r_q=rq, r_u=ru, r_fl=rfl)
        mesh.assemble_condensed(u_, q, uh_, K=K_, R=R_)
        mesh.back_substitute(duh_, du_, dq_)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        flush.zero_()
        step(u, uh, duh)
    barrier()
    mesh.profile_reset()
    mesh.profile_enable(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            flush.zero_()
            step(u, uh, duh)
        ev1.record(stream)
        barrier()
    mesh.profile_enable(False)
    ms = ev0.elapsed_time(ev1)
    prof = mesh.profile_read()
    status = mesh.element_status()
    # end to end through the public API with host buffers
    pin = lambda a: torch.as_tensor(a, dtype=f64).pin_memory()
    hu, huh, hduh = pin(st.u), pin(st.uhat), pin(st.duhat)
    hK = torch.empty(K.shape, dtype=f64).pin_memory()
    hR = torch.empty(R.shape, dtype=f64).pin_memory()
    hdu = torch.empty(du.shape, dtype=f64).pin_memory()
    hdq = torch.empty(dq.shape, dtype=f64).pin_memory()
    du_in, uh_in, duh_in = torch.empty_like(u), torch.empty_like(uh), torch.empty_like(duh)
    # Results go to the host on a copy stream while the next step computes: two sets of
    # device outputs alternate when HBM has room for the second (every copy of every
    # step still lies inside the timed region: the end event waits for the copy stream)
    outs_bytes = sum(t.numel() * t.element_size() for t in (K, R, du, dq))
    sets = [(K, R, du, dq)]
    if torch.cuda.mem_get_info(dev)[0] > 2 * outs_bytes + (4 << 30):
        sets.append(tuple(torch.empty_like(t) for t in (K, R, du, dq)))
    cstream = torch.cuda.Stream(dev)
    copied = [None] * len(sets)

    def e2e_step(n):
        k = n % len(sets)
        if copied[k] is not None:
            stream.wait_event(copied[k])            # the set's previous copy to the host is done
        du_in.copy_(hu, non_blocking=True)
        uh_in.copy_(huh, non_blocking=True)
        duh_in.copy_(hduh, non_blocking=True)
        step(du_in, uh_in, duh_in, sets[k])
        ready = torch.cuda.Event()
        ready.record(stream)
        with torch.cuda.stream(cstream):
            cstream.wait_event(ready)
            for h_, d_ in zip((hK, hR, hdu, hdq), sets[k]):
                h_.copy_(d_, non_blocking=True)
            copied[k] = torch.cuda.Event()
            copied[k].record(cstream)

    e2e_step(0)
    stream.wait_stream(cstream)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for n in range(args.steps):
        flush.zero_()
        e2e_step(n)
    stream.wait_stream(cstream)
    e1.record(stream)
    barrier()
    ms_e2e = e0.elapsed_time(e1)
    del sets
    h2d = sum(t.numel() * t.element_size() for t in (hu, huh, hduh))
    d2h = sum(t.numel() * t.element_size() for t in (hK, hR, hdu, hdq))

    # the FP64 handle and the step buffers are released before the other legs (the
    # largest workload, p=4 24^3, does not fit twice in HBM); K, R, du, dq stay for the
    # error of the mixed form
    mesh.close()
    del q, rq, ru, rfl, du_in, uh_in, duh_in, hu, huh, hduh, hK, hR, hdu, hdq
    torch.cuda.empty_cache()
    mixed = None if args.no_mixed else run_mixed(args, wl, None, dev, step_outputs=(K, R, du, dq),
                                                   inputs=(u, uh, duh), flush=flush, barrier=barrier)
    low = {}
    if not args.no_mixed and not args.no_low_precision:
        for prec, key, flags in ((2, "mixed_tf32", 0), (3, "mixed_bf16", 0), (1, "mixed_mass_scaled", 1),
                                 (2, "mixed_tf32_mass_scaled", 1), (3, "mixed_bf16_mass_scaled", 1)):
            low[key] = run_mixed(args, wl, None, dev, step_outputs=(K, R, du, dq), inputs=(u, uh, duh),
                                 flush=flush, barrier=barrier, precision=prec, flags=flags)
    # mixed orders: one GPU only (the leg takes a few minutes; scaling runs skip it)
    mixed_orders = None
    del K, R, du, dq
    torch.cuda.empty_cache()
    if world == 1 and not args.no_mixed_orders:
        mixed_orders = run_mixed_orders(args, dev, flush)
    extras = run_extras(args, dev) if (world == 1 and not args.no_extras) else None
    from paper_1605_01020_gb300.dist import max_over_ranks
    ms, ms_e2e = max_over_ranks([ms, ms_e2e], dev)
    for r in [mixed] + list(low.values()):
        if r is not None:
            (r["ms_total"],) = max_over_ranks([r["ms_total"]], dev)
    if rank != 0:
        return
    total_elems = E * args.steps * world
    value = total_elems / (ms / 1e3)
    value_e2e = total_elems / (ms_e2e / 1e3)
    clocks = clk.summary()
    # roofline of the dominant kernel (largest summed device time)
    top = max(prof.items(), key=lambda kv: kv[1][1])
    name, (launches, kms) = top
    tot_ms = sum(v[1] for v in prof.values())
    props = torch.cuda.get_device_properties(dev)
    sm_max = clocks["sm_max_mhz"] or 2070.0
    up = unit_peaks()
    peak_alu = props.multi_processor_count * DFMA_PER_CLK_PER_SM * 2 * sm_max * 1e6
    peak_src = (f"FP64 DFMA: {props.multi_processor_count} SMs x {DFMA_PER_CLK_PER_SM} FMA/clk x 2 x {sm_max:.0f} MHz "
                f"(derived)")
    if up.get("dfma_tflops"):
        peak_alu = up["dfma_tflops"] * 1e12
        peak_src = (f"FP64 DFMA, measured: {up['dfma_tflops']} TFLOP/s (profiles/peaks_gb300.txt; derived "
                    f"{props.multi_processor_count * DFMA_PER_CLK_PER_SM * 2 * sm_max * 1e6 / 1e12:.3f})")
    nq1 = wl.mesh.p + 2
    flops = {"lu_schur": a6_flops(m * Np, m * mesh.Nb) * E,
             "assemble": a4a5_flops(d, wl.mesh.p, nq1) * E}
    actual = {"lu_schur": flops["lu_schur"], "assemble": assemble_actual_flops(d, wl.mesh.p, nq1) * E}
    tpe = traffic_record("lu_schur", "fp64", (d, wl.mesh.p))
    traffic = {"lu_schur": tpe * E if tpe is not None else None}
    roof = None
    if name in flops:
        t_launch = kms / launches / 1e3
        achieved = flops[name] / t_launch
        roof = {"kernel": name, "bound": "alu", "achieved": achieved / 1e12, "peak": peak_alu / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak_alu, "traffic": traffic.get(name),
                "peak_source": peak_src,
                "algorithmic_flops_per_launch": flops[name],
                "actual_flops_per_launch": actual[name],
                "frac_actual": actual[name] / t_launch / peak_alu}
    for r in [mixed] + list(low.values()):
        if r is not None:
            mms = r.pop("ms_total")
            r["value"] = total_elems / (mms / 1e3)
            r["ms_per_step"] = mms / args.steps
            r["speedup_vs_fp64"] = ms / mms
    peaks, src = measured_peaks()
    cpu = None
    if not args.no_cpu_baseline:
        n, secs, procs = oracle_sample(wl, args.cpu_budget)
        cpu = {"value": n / secs, "unit": "elements/s", "cores": procs, "kind": "oracle",
               "sample": f"first {n} of {E} elements ({secs:.1f} s) over {procs} single-threaded worker processes "
                         f"(one per host core), numpy/scipy FP64 oracle, q-eliminated form: lifting, residual, "
                         f"condensation, back-substitution"}
    line = {"metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(wl), "elements": E, "order": wl.mesh.p, "precision": "fp64",
                       "l2": "flushed between steps (512 MB write); per-step workspace 12 GB >> L2",
                       "per_rank_elements": E, "schedule": schedule, "autotune_ms": timings64},
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": value_e2e, "unit": "elements/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "overlap": "results copied to pinned host memory on a second stream during the next step"},
            "clocks": clocks, "gpu_launches": sum(v[0] for v in prof.values()),
            "kernels": {k: {"launches": v[0], "ms": v[1], "share": v[1] / tot_ms if tot_ms else None}
                        for k, v in prof.items()},
            "element_status_nonzero": int((status != 0).sum()),
            "mixed": mixed,
            **low,
            "mixed_orders": mixed_orders,
            "extras": extras,
            "peaks": {"source": src, **{k: v for k, v in peaks.items() if isinstance(v, (int, float))}}}
    print(json.dumps(line), flush=True)


MIXED_FORMS = {1: "FP32 element matrix + partial LU, FP64 refinement",
               2: "FP32 element matrix + partial LU, Schur complement with TF32 operands on the tensor cores, "
                  "FP64 refinement",
               3: "FP32 element matrix + partial LU, Schur complement with BF16 operands on the tensor cores, "
                  "FP64 refinement"}


def run_mixed(args, wl, mesh64, dev, step_outputs, inputs, flush, barrier, precision=1, flags=0):
    """The same step in a mixed form (FP32 element matrix and partial LU, FP64
    residuals and refinement of R, du, dq; precision 2 / 3: the Schur complement with
    TF32 / BF16 operands), timed the same way; errors against the FP64 path's outputs
    on the same inputs."""
    import torch
    from paper_1605_01020_gb300 import iedg
    K64, R64, du64, dq64 = step_outputs
    u, uh, duh = inputs
    mesh = iedg.mesh_from_workload(wl, precision=precision, flags=flags)
    E, Np, m, d, T = mesh.E, mesh.Np, mesh.m, mesh.d, mesh.T
    f64 = torch.float64
    schedule, timings = None, {}
    if args.mixed_lu_tensor is not None and precision == 1:
        mesh.set_schedule(lu_tensor=args.mixed_lu_tensor)
        schedule = mesh.get_schedule()
    elif not args.no_autotune:
        from paper_1605_01020_gb300 import autotune
        qt = torch.as_tensor(wl.state.q, dtype=f64, device=dev)
        schedule, timings = autotune.autotune(mesh, u, qt, uh, precision, reps=1)
        del qt
    q = torch.empty(E, Np, m, d, dtype=f64, device=dev)
    rq, ru, rfl = torch.empty_like(q), torch.empty(E, Np, m, dtype=f64, device=dev), torch.empty(T, m, dtype=f64, device=dev)
    K, R = torch.empty_like(K64), torch.empty_like(R64)
    du, dq = torch.empty_like(du64), torch.empty_like(dq64)

    def step():
        mesh.eval_residual(u, uh, q=None, q_out=q, r_q=rq, r_u=ru, r_fl=rfl)
        mesh.assemble_condensed(u, q, uh, K=K, R=R)
        mesh.back_substitute(duh, du, dq)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    barrier()
    mesh.profile_reset()
    mesh.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        flush.zero_()
        step()
    e1.record()
    barrier()
    mesh.profile_enable(False)
    prof = mesh.profile_read()
    tot = sum(v[1] for v in prof.values())
    err = lambda a, b: float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))
    status = mesh.element_status()
    # the FP32 partial LU against the FP32 FMA rate (its updates and panels run on FFMA;
    # the tensor-core forms put only the deferred Schur GEMM on tcgen05)
    roof = None
    if "lu_schur" in prof:
        launches, kms = prof["lu_schur"]
        props = torch.cuda.get_device_properties(dev)
        up = unit_peaks()
        peak = props.multi_processor_count * FFMA_PER_CLK_PER_SM * 2 * 2070.0e6
        src = f"FP32 FFMA: {props.multi_processor_count} SMs x {FFMA_PER_CLK_PER_SM} FMA/clk x 2 x 2070 MHz (derived)"
        if up.get("ffma_tflops"):
            peak, src = up["ffma_tflops"] * 1e12, f"FP32 FFMA, measured: {up['ffma_tflops']} TFLOP/s"
        fl = a6_flops(m * Np, m * mesh.Nb) * E
        ach = fl / (kms / launches / 1e3)
        sched = mesh.get_schedule()
        roof = {"kernel": "lu_schur", "bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": ach / peak, "algorithmic_flops_per_launch": fl,
                "peak_source": src, "share_of_step": kms / tot if tot else None, "lu_form": sched["lu_tensor"]}
        if up.get("tf32_tcgen05_tflops") and (sched["lu_tensor"] or precision in (2, 3)):
            # the tensor-core forms against the measured TF32 tcgen05 rate (the FP32 form
            # issues three TF32 products per trailing-update flop: 3xTF32)
            tp = up["tf32_tcgen05_tflops"] * 1e12
            roof["tensor"] = {"bound": "tensor", "peak": tp / 1e12, "unit": "TFLOP/s",
                              "frac_algorithmic": ach / tp,
                              "peak_source": f"tcgen05 kind::tf32, measured: {up['tf32_tcgen05_tflops']} TFLOP/s"}
    out = {"ms_total": e0.elapsed_time(e1),
           "precision": MIXED_FORMS[precision] + ("; element systems scaled by the mass matrix's inverse Cholesky "
                                                  "factor before the factorisation" if flags else ""),
           "schedule": schedule, "autotune_ms": timings, "roofline": roof,
           "err_vs_fp64": {"K": err(K, K64), "R": err(R, R64), "du": err(du, du64), "dq": err(dq, dq64)},
           "element_status_nonzero": int((status != 0).sum()),
           "gpu_launches": sum(v[0] for v in prof.values()),
           "kernels": {k: {"launches": v[0], "ms": v[1], "share": v[1] / tot if tot else None} for k, v in prof.items()}}
    mesh.close()
    return out


def run_mixed_orders(args, dev, flush):
    """Mixed-order batch (3D, p in {2,3,4} by seed, 8192 elements): the same step on a
    mesh whose elements have different orders, FP64 and mixed-precision forms.  Each
    form is autotuned, captured once in a CUDA graph and timed by graph replays; the
    kernel breakdown comes from one profiled eager step."""
    import torch
    from paper_1605_01020_gb300 import iedg
    from paper_1605_01020_gb300 import workloads as W
    t0 = time.perf_counter()
    wl = W.config(4, N=args.mo_cells)
    msh, st, prm = wl.mesh, wl.state, wl.params
    t_build = time.perf_counter() - t0
    f64 = torch.float64
    cat = lambda xs: torch.as_tensor(np.ascontiguousarray(np.concatenate(xs)), dtype=f64, device=dev)
    u, qin = cat(st.u), cat(st.q)
    uh = torch.as_tensor(st.uhat, dtype=f64, device=dev)
    duh = torch.as_tensor(st.duhat, dtype=f64, device=dev)
    E, m, d = msh.n_elem, msh.d + 2, msh.d
    nbe = np.array([len(t) for t in msh.elem_trace])
    lu_flops = float(sum(a6_flops(m * (int(p) + 1) ** 3, m * int(nb)) for p, nb in zip(msh.orders, nbe)))
    res = {"workload": wl.name, "elements": E,
           "orders": {str(p): int((msh.orders == p).sum()) for p in (2, 3, 4)},
           "n_trace": msh.n_trace, "mesh_build_s": t_build,
           "lu_algorithmic_flops_per_launch": lu_flops}
    outs = {}
    for precision in (0, 1):
        mesh = iedg.MixedOrderMesh(msh.node_xyz, msh.elem_trace, msh.n_trace, msh.orders, msh.face_degree,
                                   gamma=prm["gamma"], Pr=prm["Pr"], Re=prm["Re"], Minf=prm["Minf"],
                                   alpha=prm["alpha"], precision=precision)
        schedule, timings = None, {}
        if not args.no_autotune:
            from paper_1605_01020_gb300 import autotune
            schedule, timings = autotune.autotune(mesh, u, qin, uh, precision, reps=1)
        q = torch.empty(mesh._qshape, dtype=f64, device=dev)
        rq, dq = torch.empty_like(q), torch.empty_like(q)
        ru, du = torch.empty(mesh._ushape, dtype=f64, device=dev), torch.empty(mesh._ushape, dtype=f64, device=dev)
        rfl = torch.empty(mesh.T, m, dtype=f64, device=dev)
        K = torch.empty(mesh.nnzb, m, m, dtype=f64, device=dev)
        R = torch.empty(mesh.T, m, dtype=f64, device=dev)

        def step():
            mesh.eval_residual(u, uh, q=None, q_out=q, r_q=rq, r_u=ru, r_fl=rfl)
            mesh.assemble_condensed(u, q, uh, K=K, R=R)
            mesh.back_substitute(duh, du, dq)

        for _ in range(args.warmup):
            flush.zero_()
            step()
        torch.cuda.synchronize()
        mesh.profile_reset()
        mesh.profile_enable(True)
        step()
        mesh.profile_enable(False)
        prof = mesh.profile_read()
        launches_per_step = sum(v[0] for v in prof.values())
        # one step captured in a CUDA graph, timed by replays
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            step()
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step()
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        status = mesh.element_status()
        tot = sum(v[1] for v in prof.values())
        lu = prof.get("lu_schur", (1, float("nan")))
        r = {"schedule": schedule, "autotune_ms": timings, "value": E * args.steps / (ms / 1e3),
             "unit": "elements/s", "ms_per_step": ms / args.steps, "timing": "CUDA graph replay of one step",
             "gpu_launches_per_step": launches_per_step,
             "element_status_nonzero": int((status != 0).sum()),
             "lu_schur_ms": lu[1] / lu[0], "lu_schur_tflops": lu_flops / (lu[1] / lu[0] / 1e3) / 1e12,
             "kernels": {k: {"launches": v[0], "ms": v[1], "share": v[1] / tot if tot else None}
                         for k, v in prof.items()}}
        outs[precision] = [t.clone() for t in (K, R, du, dq)]
        res["fp64" if precision == 0 else "mixed"] = r
        del g
        mesh.close()
    err = lambda a, b: float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))
    res["mixed"]["err_vs_fp64"] = {k: err(a, b) for k, a, b in zip(("K", "R", "du", "dq"), outs[1], outs[0])}
    res["mixed"]["speedup_vs_fp64"] = res["fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"]
    return res


def run_extras(args, dev):
    """Measurements of the rows beyond the condensation itself, each on its own small
    workload: the Roe-type stabilisation (assembly + condensation of the 3D p=3 16^3
    workload in FP64, against Lax-Friedrichs on the same handle type), the trace
    solve (GMRES with block Jacobi and with BILU(0), 3D p=3 8^3), and one DIRK(3,3)
    time step with Newton per stage (2D p=2 8x8)."""
    import torch
    from paper_1605_01020_gb300 import iedg, timestep
    from paper_1605_01020_gb300 import workloads as W
    f64 = torch.float64
    out = {}
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    # Roe vs Lax-Friedrichs, one assemble_condensed call each (median of 3 after 2 warm-ups)
    wl = W.config(2, N=args.cells)
    st = wl.state
    u, q, uh = (torch.as_tensor(a, dtype=f64, device=dev) for a in (st.u, st.q, st.uhat))
    for name, stab in (("lax_friedrichs", 0), ("roe", 1)):
        mesh = iedg.mesh_from_workload(W.Workload(wl.name, wl.mesh, st, dict(wl.params, stab=stab)))
        K = torch.empty(mesh.nnzb, mesh.m, mesh.m, dtype=f64, device=dev)
        R = torch.empty(mesh.T, mesh.m, dtype=f64, device=dev)
        ts = []
        for i in range(5):
            a0, a1 = ev()
            a0.record()
            mesh.assemble_condensed(u, q, uh, K=K, R=R)
            a1.record()
            torch.cuda.synchronize()
            if i >= 2:
                ts.append(a0.elapsed_time(a1))
        out[f"assemble_condensed_{name}"] = {"ms": statistics.median(ts), "elements": mesh.E,
                                             "elements_per_s": mesh.E / (statistics.median(ts) / 1e3)}
        mesh.close()
    del u, q, uh, K, R
    torch.cuda.empty_cache()
    # trace solve on the condensed K of the 8^3 case
    wl = W.config(2, N=8)
    st = wl.state
    mesh = iedg.mesh_from_workload(wl)
    u, q, uh = (torch.as_tensor(a, dtype=f64, device=dev) for a in (st.u, st.q, st.uhat))
    K, R = mesh.assemble_condensed(u, q, uh)
    for name, kind in (("block_jacobi", iedg.PREC_BLOCK_JACOBI), ("bilu0", iedg.PREC_BILU0)):
        mesh.set_trace_precond(kind)
        mesh.trace_solve(K, R, rtol=1e-10, max_iter=3000)             # warm-up (colouring on first use)
        t0 = time.perf_counter()
        dU, its, rr = mesh.trace_solve(K, R, rtol=1e-10, max_iter=3000)
        torch.cuda.synchronize()
        out[f"trace_solve_{name}"] = {"ms": 1e3 * (time.perf_counter() - t0), "iterations": its,
                                      "rel_residual": rr, "trace_nodes": mesh.T,
                                      "workload": "3D p=3 8^3 condensed K, rtol 1e-10, restart 30"}
    mesh.close()
    del u, q, uh, K, R
    torch.cuda.empty_cache()
    # one DIRK(3,3) step, Newton per stage, minimal-residual guess from the 3rd step on
    wl = W.config(1)
    st = W.make_state(wl.mesh, W.fourier_perturbed_field(2, 0.2, 41, amp=0.05), 42, noise=0.005)
    mesh = iedg.mesh_from_workload(wl)
    u = torch.as_tensor(st.u, dtype=f64, device=dev)
    uh = torch.as_tensor(st.uhat, dtype=f64, device=dev)
    q = mesh.eval_residual(u, uh, q=None)["q"]
    stepper = timestep.Stepper(mesh, 0.005, newton_tol=1e-10)
    state = (u, q, uh)
    times = []
    for n in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        state = stepper.step(*state, use_mr=True)[:3]
        torch.cuda.synchronize()
        times.append(1e3 * (time.perf_counter() - t0))
    out["dirk33_step"] = {"ms_per_step": statistics.median(times[1:]), "newton_iterations": stepper.newton_iters,
                          "workload": "2D p=2 8x8, dt = 0.005, Newton to 1e-10, GMRES + block Jacobi"}
    mesh.close()
    # the same on the 3D Taylor-Green vortex (config 2's recipe on 8^3 cells, p = 3)
    wl = W.config(2, N=8)
    st = wl.state
    mesh = iedg.mesh_from_workload(wl)
    u = torch.as_tensor(st.u, dtype=f64, device=dev)
    uh = torch.as_tensor(st.uhat, dtype=f64, device=dev)
    q = mesh.eval_residual(u, uh, q=None)["q"]
    stepper = timestep.Stepper(mesh, 0.005, newton_tol=1e-10)
    state = (u, q, uh)
    times = []
    for n in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        state = stepper.step(*state, use_mr=True)[:3]
        torch.cuda.synchronize()
        times.append(1e3 * (time.perf_counter() - t0))
    out["dirk33_step_tgv3d"] = {"ms_per_step": statistics.median(times[1:]), "newton_iterations": stepper.newton_iters,
                                "elements": mesh.E,
                                "workload": "3D Taylor-Green p=3 8^3 (config 2 field, Re 2.5e5), dt = 0.005, "
                                            "Newton to 1e-10, GMRES + block Jacobi"}
    mesh.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--cells", type=int, default=None, help="override cells per direction (smaller case)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision measurement")
    ap.add_argument("--no-low-precision", action="store_true",
                    help="skip the mixed forms with TF32 / BF16 Schur operands")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch schedule")
    ap.add_argument("--no-mixed-orders", action="store_true", help="skip the mixed-order batch (p in {2,3,4})")
    ap.add_argument("--no-extras", action="store_true", help="skip the Roe / trace-solve / DIRK measurements")
    ap.add_argument("--mo-cells", type=int, default=None, help="mixed-order batch: N x N x 2N cells (default 16)")
    ap.add_argument("--mixed-lu-tensor", type=int, default=None, choices=[0, 1, 2],
                    help="mixed FP32 form: fixed LU form instead of the autotuner's choice (0 FFMA updates, "
                         "1 deferred Schur complement on tcgen05, 2 every trailing update on tcgen05)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-elems", type=int, default=2, help="reference arm: elements per core per step")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_1605_01020_gb300 import workloads as W
    wl = W.config(args.config, N=args.cells)
    if args.impl == "reference":
        run_reference(args, wl, rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    run_ours(args, wl, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
