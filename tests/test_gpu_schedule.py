"""Launch schedules (persistent vs one-CTA-per-element LU, LU panel width, assembly
column chunk) give the same condensed system, and the autotuner picks and caches
one of them."""
import json

import numpy as np
import pytest

from paper_1605_01020_gb300 import workloads as W
from gpu_helpers import dev, host, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_schedules_agree(precision):
    from paper_1605_01020_gb300 import autotune, iedg
    wl = W.config(2, N=3)
    st = wl.state
    mesh = iedg.mesh_from_workload(wl, precision=precision)
    u, q, uh = dev(st.u), dev(st.q), dev(st.uhat)
    ref = None
    for cand in autotune.candidates(precision, mesh.order):
        mesh.set_schedule(**cand)
        assert mesh.get_schedule() == cand
        K, R = mesh.assemble_condensed(u, q, uh)
        du, dq = mesh.back_substitute(dev(st.duhat))
        out = [host(t) for t in (K, R, du, dq)]
        if ref is None:
            ref = out
            continue
        tol = 1e-11 if precision == 0 else 1e-4          # FP32 K: FFMA vs 3xTF32 tensor-core updates
        assert rel_err(out[0], ref[0]) <= tol, cand
        for a, b in zip(out[1:], ref[1:]):
            assert rel_err(a, b) <= 1e-10, cand


def test_autotune_picks_and_caches(tmp_path):
    from paper_1605_01020_gb300 import autotune, iedg
    wl = W.config(2, N=3)
    st = wl.state
    mesh = iedg.mesh_from_workload(wl)
    u, q, uh = dev(st.u), dev(st.q), dev(st.uhat)
    cache = tmp_path / "sched.json"
    best, timings = autotune.autotune(mesh, u, q, uh, 0, reps=1, cache_path=str(cache))
    assert best in autotune.candidates(0, mesh.order)
    assert len(timings) == len(autotune.candidates(0, mesh.order))
    assert mesh.get_schedule() == best
    data = json.loads(cache.read_text())
    assert list(data.values())[0]["schedule"] == best
    # second call comes from the cache
    best2, _ = autotune.autotune(mesh, u, q, uh, 0, reps=1, cache_path=str(cache))
    assert best2 == best


def test_bad_schedule_rejected():
    from paper_1605_01020_gb300 import iedg
    mesh = iedg.mesh_from_workload(W.config(1, N=2))
    with pytest.raises(iedg.IedgError):
        mesh.set_schedule(lu_panel=24)
