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


def _pair_keys(elem_trace, elems, n_trace):
    """Sorted unique keys row * n_trace + col of the trace-node pairs that share one
    of `elems` (the block pattern those elements produce, row-major)."""
    if len(elems) == 0:
        return np.zeros(0, dtype=np.int64)
    if isinstance(elem_trace, list):
        keys = [(np.asarray(elem_trace[e], dtype=np.int64)[:, None] * n_trace +
                 np.asarray(elem_trace[e], dtype=np.int64)[None, :]).ravel() for e in elems]
        return np.unique(np.concatenate(keys))
    tr = np.asarray(elem_trace, dtype=np.int64)[elems]
    return np.unique((tr[:, :, None] * n_trace + tr[:, None, :]).ravel())


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

    Every pattern is held as sorted pair keys row * n_trace + col, so the block index
    of a pair inside a CSR pattern is its position in that pattern's key array.
    """

    def __init__(self, elem_trace, n_trace, parts, rank, world):
        parts = np.asarray(parts, dtype=np.int64)
        n = self.n_trace = int(n_trace)
        self.rank, self.world = rank, world
        self.elems = np.nonzero(parts == rank)[0]
        by_rank = [np.nonzero(parts == r)[0] for r in range(world)]
        # owner of every trace node: the lowest rank among the elements touching it
        if isinstance(elem_trace, list):
            flat = np.concatenate([np.asarray(t, dtype=np.int64) for t in elem_trace]) if len(elem_trace) else \
                np.zeros(0, dtype=np.int64)
            eparts = np.repeat(parts, [len(t) for t in elem_trace])
        else:
            et = np.asarray(elem_trace, dtype=np.int64)
            flat, eparts = et.ravel(), np.repeat(parts, et.shape[1] if et.ndim == 2 else 0)
        owner = np.full(n, world, dtype=np.int64)
        np.minimum.at(owner, flat, eparts)
        self.owner = owner
        self.touch = [np.unique(flat[eparts == r]) for r in range(world)]
        self.l2g = self.touch[rank]
        self.local_elem_trace = [np.searchsorted(self.l2g, np.asarray(elem_trace[e], dtype=np.int64))
                                 for e in self.elems]
        if not isinstance(elem_trace, list) and len(self.local_elem_trace):
            self.local_elem_trace = np.stack(self.local_elem_trace)
        # patterns of every rank's elements over global ids
        keys = [_pair_keys(elem_trace, by_rank[r], n) for r in range(world)]
        mine = keys[rank]
        self.row_ptr_local = np.zeros(len(self.l2g) + 1, dtype=np.int64)
        self.row_ptr_local[1:] = np.cumsum(np.bincount(np.searchsorted(self.l2g, mine // n),
                                                       minlength=len(self.l2g)))
        self.col_local = np.searchsorted(self.l2g, mine % n).astype(np.int64)
        # owned rows over the union of every rank's columns
        union = np.unique(np.concatenate(keys)) if world else np.zeros(0, dtype=np.int64)
        full = [union[owner[union // n] == r] for r in range(world)]
        self.owned = np.nonzero(owner == rank)[0]
        own = full[rank]
        self.row_ptr = np.zeros(len(self.owned) + 1, dtype=np.int64)
        self.row_ptr[1:] = np.cumsum(np.bincount(np.searchsorted(self.owned, own // n),
                                                 minlength=len(self.owned)))
        self.col = (own % n).astype(np.int64)
        self._plan(keys, full)

    def _plan(self, keys, full):
        """Where each block and row goes: this rank's own contributions, what it sends to
        every owner (in its local row-major order) and where what it receives lands."""
        world, rank, n, owner = self.world, self.rank, self.n_trace, self.owner
        mine = keys[rank]
        o_blk = owner[mine // n]
        self.own_blocks_src = np.nonzero(o_blk == rank)[0]
        self.own_blocks_dst = np.searchsorted(full[rank], mine[self.own_blocks_src])
        self.send_blocks = [np.nonzero(o_blk == q)[0] if q != rank else np.zeros(0, dtype=np.int64)
                            for q in range(world)]
        o_row = owner[self.l2g]
        self.own_rows_src = np.nonzero(o_row == rank)[0]
        self.own_rows_dst = np.searchsorted(self.owned, self.l2g[self.own_rows_src])
        self.send_rows = [np.nonzero(o_row == q)[0] if q != rank else np.zeros(0, dtype=np.int64)
                          for q in range(world)]
        # what this rank receives from each sender, in the sender's order
        self.recv_blocks_dst = [np.zeros(0, dtype=np.int64) for _ in range(world)]
        self.recv_rows_dst = [np.zeros(0, dtype=np.int64) for _ in range(world)]
        for s in range(world):
            if s == rank:
                continue
            ks = keys[s][owner[keys[s] // n] == rank]
            self.recv_blocks_dst[s] = np.searchsorted(full[rank], ks)
            rows = self.touch[s][owner[self.touch[s]] == rank]
            self.recv_rows_dst[s] = np.searchsorted(self.owned, rows)
        # halo of the trace increments: owned values each peer needs, and where the
        # values this rank needs come from
        self.halo_send = [np.nonzero(np.isin(self.owned, self.touch[q]))[0].astype(np.int64) if q != rank
                          else np.zeros(0, dtype=np.int64) for q in range(world)]
        self.halo_recv = [np.nonzero(o_row == q)[0].astype(np.int64) for q in range(world)]

    # ------------------------------------------------------------------ exchange
    def _exchange(self, payload_send, recv_shapes, like):
        """Point-to-point: payload_send[q] to rank q, returns the tensors received from
        every other rank.  All sends and receives of the step are issued as one batch
        (batch_isend_irecv), so backends that serialise point-to-point operations per
        peer (NCCL) cannot deadlock on the order in which ranks post them."""
        import torch
        import torch.distributed as dist
        ops, recvs = [], [None] * self.world
        for q in range(self.world):
            if q == self.rank:
                continue
            if recv_shapes[q][0] > 0:
                recvs[q] = torch.empty(recv_shapes[q], dtype=like.dtype, device=like.device)
                ops.append(dist.P2POp(dist.irecv, recvs[q], q))
            if payload_send[q] is not None and payload_send[q].shape[0] > 0:
                ops.append(dist.P2POp(dist.isend, payload_send[q].contiguous(), q))
        if ops:
            for r in dist.batch_isend_irecv(ops):
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
