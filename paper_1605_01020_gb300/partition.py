"""One mesh split over several ranks: the exchange step of the condensed system.

The element-local work (Sec. 2.2.1: fluxes, element blocks, partial LU, Eq. LS) needs
only an element's own data and the trace values of its slots, so each rank runs the
library on the elements it owns, numbered with local trace ids.  The condensed
matrix and right-hand side are sums over elements (K = sum_e P_e^T K_e P_e, block
rows per trace node, Sec. 2.2.2), so a trace node on a partition interface receives
contributions from every rank whose elements touch it.  That is the one exchange
step: every rank sends the block rows of the interface nodes it does not own to their
owner (the lowest rank touching the node), which adds them to its own.  After the
global trace solve the owners send the increments of those nodes back (halo), so
each rank can back-substitute its elements.

Everything here is host bookkeeping plus point-to-point sends of torch tensors: it
runs with any torch.distributed backend (NCCL between GPUs, gloo on CPU for tests)
and never touches the element arithmetic.  The plan is built from the global mesh on
every rank, without communication, so senders and receivers agree on the order of
the blocks they exchange.
"""
import numpy as np


def _row_patterns(elem_trace, elems):
    """Sorted column sets (global trace ids) of the block rows touched by `elems`."""
    rows = {}
    for e in elems:
        tr = np.unique(np.asarray(elem_trace[e], dtype=np.int64))
        for t in tr.tolist():
            rows.setdefault(t, set()).update(tr.tolist())
    return {t: np.array(sorted(c), dtype=np.int64) for t, c in rows.items()}


class Partition:
    """Plan of the exchange for one rank.

    elem_trace: per element, the global trace ids of its slots (array [E][Nb] or a list
    of arrays for meshes of mixed orders); n_trace: global trace-node count; parts:
    rank of every element; rank, world: this rank and the number of ranks.

    Attributes: elems (global ids of the local elements, increasing), l2g (global id of
    each local trace node, increasing), local_elem_trace (slots in local ids, for the
    library's mesh of the local elements), owned (global ids of the nodes this rank
    owns, increasing), row_ptr / col (block-compressed pattern of the owned rows over
    global column ids, columns sorted), and the local pattern row_ptr_local /
    col_local the library produces for the local mesh (same rule: sorted local
    columns, one block per pair of trace nodes sharing an element).
    """

    def __init__(self, elem_trace, n_trace, parts, rank, world):
        parts = np.asarray(parts, dtype=np.int64)
        E = len(parts)
        self.rank, self.world, self.n_trace = rank, world, int(n_trace)
        self.elems = np.nonzero(parts == rank)[0]
        # owner of every trace node: the lowest rank among the elements touching it
        owner = np.full(self.n_trace, world, dtype=np.int64)
        touch = [set() for _ in range(world)]
        for e in range(E):
            tr = np.asarray(elem_trace[e], dtype=np.int64)
            owner[tr] = np.minimum(owner[tr], parts[e])
            touch[parts[e]].update(tr.tolist())
        self.owner = owner
        self.touch = [np.array(sorted(s), dtype=np.int64) for s in touch]
        self.l2g = self.touch[rank]
        g2l = {g: i for i, g in enumerate(self.l2g.tolist())}
        self.local_elem_trace = [np.array([g2l[t] for t in np.asarray(elem_trace[e]).tolist()], dtype=np.int64)
                                 for e in self.elems]
        if not isinstance(elem_trace, list) and len(self.local_elem_trace):
            self.local_elem_trace = np.stack(self.local_elem_trace)
        # patterns: rows of each rank over global columns
        pats = [_row_patterns(elem_trace, np.nonzero(parts == r)[0]) for r in range(world)]
        mine = pats[rank]
        self.row_ptr_local = np.zeros(len(self.l2g) + 1, dtype=np.int64)
        cols_local = []
        for i, g in enumerate(self.l2g.tolist()):
            cg = mine[g]
            cols_local.append(np.array([g2l[c] for c in cg.tolist()], dtype=np.int64))
            self.row_ptr_local[i + 1] = self.row_ptr_local[i] + len(cg)
        self.col_local = np.concatenate(cols_local) if cols_local else np.zeros(0, dtype=np.int64)
        # owned rows over the union of every rank's columns
        self.owned = np.nonzero(owner == rank)[0]
        full = {}
        for r in range(world):
            for g, cg in pats[r].items():
                if owner[g] == rank:
                    full.setdefault(g, set()).update(cg.tolist())
        self.row_ptr = np.zeros(len(self.owned) + 1, dtype=np.int64)
        cols = []
        for i, g in enumerate(self.owned.tolist()):
            cg = np.array(sorted(full[g]), dtype=np.int64)
            cols.append(cg)
            self.row_ptr[i + 1] = self.row_ptr[i] + len(cg)
        self.col = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
        # where each rank's local blocks land: for rank r and each block of its local
        # pattern (row-major), the owner and the block's index in the owner's owned rows
        self._plan(pats, owner)

    def _owned_index(self, r, pats, owner):
        """For an owner rank r: {global row: (offset of the row, {global col: slot})}."""
        out = {}
        off = 0
        full = {}
        for q in range(self.world):
            for g, cg in pats[q].items():
                if owner[g] == r:
                    full.setdefault(g, set()).update(cg.tolist())
        for g in sorted(full):
            cg = sorted(full[g])
            out[g] = (off, {c: k for k, c in enumerate(cg)})
            off += len(cg)
        return out

    def _plan(self, pats, owner):
        world, rank = self.world, self.rank
        idx = [self._owned_index(r, pats, owner) for r in range(world)]
        # blocks and rows this rank sends to each owner (in its local row-major order)
        self.send_blocks = [[] for _ in range(world)]   # local block ids
        self.send_rows = [[] for _ in range(world)]     # local row ids
        # blocks and rows of this rank's own contributions to its owned rows
        self.own_blocks_src, self.own_blocks_dst = [], []
        self.own_rows_src, self.own_rows_dst = [], []
        row_of_owned = {g: i for i, g in enumerate(self.owned.tolist())}
        for i, g in enumerate(self.l2g.tolist()):
            o = int(owner[g])
            off, slots = idx[o][g]
            lo, hi = self.row_ptr_local[i], self.row_ptr_local[i + 1]
            for k in range(lo, hi):
                cg = int(self.l2g[self.col_local[k]])
                if o == rank:
                    self.own_blocks_src.append(k)
                    self.own_blocks_dst.append(off + slots[cg])
                else:
                    self.send_blocks[o].append(k)
            if o == rank:
                self.own_rows_src.append(i)
                self.own_rows_dst.append(row_of_owned[g])
            else:
                self.send_rows[o].append(i)
        # what this rank receives from each sender, in the sender's order
        self.recv_blocks_dst = [[] for _ in range(world)]
        self.recv_rows_dst = [[] for _ in range(world)]
        mine = idx[rank]
        row_of_owned = {g: i for i, g in enumerate(self.owned.tolist())}
        for s in range(world):
            if s == rank:
                continue
            l2g_s = self.touch[s]
            ps = pats[s]
            for g in l2g_s.tolist():                       # sender's local rows, increasing
                if int(owner[g]) != rank:
                    continue
                off, slots = mine[g]
                for cg in ps[g].tolist():                  # sender's sorted columns of the row
                    self.recv_blocks_dst[s].append(off + slots[cg])
                self.recv_rows_dst[s].append(row_of_owned[g])
        # halo of the trace increments: owned values each peer needs, and where the
        # values this rank needs come from
        self.halo_send = [np.nonzero(np.isin(self.owned, self.touch[q]))[0].astype(np.int64) if q != rank
                          else np.zeros(0, dtype=np.int64) for q in range(world)]
        self.halo_recv = [np.array([i for i, g in enumerate(self.l2g.tolist()) if int(owner[g]) == q],
                                   dtype=np.int64) for q in range(world)]

    # ------------------------------------------------------------------ exchange
    def _exchange(self, payload_send, recv_shapes, like):
        """Point-to-point: payload_send[q] to rank q, returns the tensors received from
        every other rank (the receives are posted before the sends complete)."""
        import torch
        import torch.distributed as dist
        reqs, recvs = [], [None] * self.world
        for q in range(self.world):
            if q == self.rank:
                continue
            if recv_shapes[q][0] > 0:
                recvs[q] = torch.empty(recv_shapes[q], dtype=like.dtype, device=like.device)
                reqs.append(dist.irecv(recvs[q], src=q))
        for q in range(self.world):
            if q == self.rank or payload_send[q] is None or payload_send[q].shape[0] == 0:
                continue
            reqs.append(dist.isend(payload_send[q].contiguous(), dst=q))
        for r in reqs:
            r.wait()
        return recvs

    def assemble_owned(self, K_local, R_local):
        """Owned block rows of the global K and R from the local ones (the library's
        output for the local mesh: K_local [nnzb_local, m, m] in the local pattern,
        R_local [n_local, m]).  Returns K_owned [len(col), m, m] over (row_ptr, col) and
        R_owned [len(owned), m]: this rank's contributions first, then every other
        rank's in rank order."""
        import torch
        dev = K_local.device
        m = K_local.shape[-1]
        K_own = torch.zeros((len(self.col), m, m), dtype=K_local.dtype, device=dev)
        R_own = torch.zeros((len(self.owned), m), dtype=R_local.dtype, device=dev)
        t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.int64), device=dev)
        K_own.index_add_(0, t(self.own_blocks_dst), K_local[t(self.own_blocks_src)])
        R_own.index_add_(0, t(self.own_rows_dst), R_local[t(self.own_rows_src)])
        sendK = [K_local[t(b)] if len(b) else None for b in self.send_blocks]
        sendR = [R_local[t(r)] if len(r) else None for r in self.send_rows]
        gotK = self._exchange(sendK, [(len(b), m, m) for b in self.recv_blocks_dst], K_local)
        gotR = self._exchange(sendR, [(len(r), m) for r in self.recv_rows_dst], R_local)
        for q in range(self.world):
            if gotK[q] is not None:
                K_own.index_add_(0, t(self.recv_blocks_dst[q]), gotK[q])
            if gotR[q] is not None:
                R_own.index_add_(0, t(self.recv_rows_dst[q]), gotR[q])
        return K_own, R_own

    def halo(self, dU_owned):
        """Trace increments of every local node (dU_owned [len(owned), m] -> [n_local, m])."""
        import torch
        dev = dU_owned.device
        m = dU_owned.shape[-1]
        t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.int64), device=dev)
        out = torch.empty((len(self.l2g), m), dtype=dU_owned.dtype, device=dev)
        mine = self.halo_recv[self.rank]
        if len(mine):
            pos = np.searchsorted(self.owned, self.l2g[mine])
            out[t(mine)] = dU_owned[t(pos)]
        send = [dU_owned[t(s)] if len(s) else None for s in self.halo_send]
        got = self._exchange(send, [(len(r), m) for r in self.halo_recv], dU_owned)
        for q in range(self.world):
            if q != self.rank and got[q] is not None:
                out[t(self.halo_recv[q])] = got[q]
        return out
