"""One mesh split over two ranks (gloo on CPU): the exchange of the interface block
rows of K and R, and the halo of the trace increments.  The element-local outputs
the library would produce on each rank are stood in for by the oracle's condensed
blocks of that rank's elements (assembled in local trace ids); after the exchange
each rank's owned rows must equal the global assembly's rows (pattern bit-exact,
values to round-off of the changed summation order), and the halo must give every
rank the increments of all its trace nodes."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _parts(kind, E):
    if kind == "slabs":
        return (np.arange(E) >= E // 2).astype(np.int64)
    return np.random.default_rng(5).integers(0, 2, E)


def _worker(rank, world, port, kind, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
        from oracle import iedg as oiedg
        from oracle_helpers import problem
        from paper_1605_01020_gb300 import workloads as W
        from paper_1605_01020_gb300.partition import Partition
        wl = W.config(1, N=4)
        st = wl.state
        mesh = wl.mesh
        E = mesh.n_elem
        parts = _parts(kind, E)
        part = Partition(mesh.elem_trace, mesh.n_trace, parts, rank, world)
        pb = problem(mesh, wl.params)
        Ke, Re = zip(*[pb.condense_qelim(int(e), st.u, st.q, st.uhat) for e in part.elems])
        rp_l, col_l, vals_l, R_l = oiedg.assemble(part.local_elem_trace, len(part.l2g), np.array(Ke), np.array(Re))
        res = {"pattern_local": bool(np.array_equal(rp_l, part.row_ptr_local) and np.array_equal(col_l, part.col_local))}
        K_own, R_own = part.assemble_owned(torch.as_tensor(vals_l), torch.as_tensor(R_l))
        # the global assembly's owned rows
        Kg, Rg = zip(*[pb.condense_qelim(e, st.u, st.q, st.uhat) for e in range(E)])
        rp_g, col_g, vals_g, R_g = oiedg.assemble(mesh.elem_trace, mesh.n_trace, np.array(Kg), np.array(Rg))
        same_pattern, kerr, scale = True, 0.0, np.abs(vals_g).max()
        for i, g in enumerate(part.owned.tolist()):
            a, b = part.row_ptr[i], part.row_ptr[i + 1]
            ga, gb = rp_g[g], rp_g[g + 1]
            same_pattern &= bool(np.array_equal(part.col[a:b], col_g[ga:gb]))
            if same_pattern:
                kerr = max(kerr, float(np.abs(K_own[a:b].numpy() - vals_g[ga:gb]).max()) / scale)
        rerr = float(np.abs(R_own.numpy() - R_g[part.owned]).max() / np.abs(R_g).max())
        res.update(pattern_owned=same_pattern, kerr=kerr, rerr=rerr, n_owned=len(part.owned),
                   n_local=len(part.l2g), n_elems=len(part.elems))
        # halo of the increments
        dU = np.random.default_rng(11).standard_normal((mesh.n_trace, pb.m))
        got = part.halo(torch.as_tensor(dU[part.owned])).numpy()
        res["halo_exact"] = bool(np.array_equal(got, dU[part.l2g]))
        out[rank] = res
    finally:
        torch.distributed.destroy_process_group()


@pytest.mark.parametrize("kind", ["slabs", "scattered"])
def test_interface_rows_and_halo_two_gloo_ranks(kind):
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), kind, out), nprocs=world, join=True)
    from paper_1605_01020_gb300 import workloads as W
    wl = W.config(1, N=4)
    assert sum(out[r]["n_owned"] for r in range(world)) == wl.mesh.n_trace     # every row owned once
    assert sum(out[r]["n_elems"] for r in range(world)) == wl.mesh.n_elem
    for r in range(world):
        res = out[r]
        assert res["pattern_local"] and res["pattern_owned"] and res["halo_exact"], res
        assert res["kerr"] <= 1e-13 and res["rerr"] <= 1e-13, res
        assert res["n_local"] > res["n_owned"] or r == 0                        # rank 1 needs halo nodes
