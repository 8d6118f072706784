"""Ghost exchange between processes that own different blocks (arxiv
2605.14780, Sec. V-B; Sec. V-A for the partition-aware coordinates).

A process owns some blocks of the grid.  Its boundary rows may read cells of
blocks other processes own; for every such remote block it receives the
*bounding box* of the cells its rows read, packed by the owner with the
library's pack kernel (``bc_pack_run``), exchanged with grouped point to
point sends and receives (NCCL on GPUs), into a local staging buffer.  Each
received box is a block of the local grid (extents of the box, no ghost
cells, the remote block's components and levels), and the rows that read
remote cells are rewritten to read the box's cells instead, so the local
plan is an ordinary plan over the owned blocks plus the staging blocks and
its apply runs the same kernels as on one GPU.

Host-side planning and argument marshalling only: packing and the ghost
fill run in the library's kernels, the transfer in the collective backend.
Cubed-sphere rows generated on the device (``BC_GEOM_CUBED_SPHERE*``) are
not partitioned here: their source cells are only known after the plan's
geometry kernel runs.
"""
from __future__ import annotations

import numpy as np

from . import bc, specs


def owners_by_cells(blocks, world):
    """Contiguous ranges of blocks per rank, balancing the data cells times
    levels times components (the work of a rank's ghost fill scales with its
    blocks' sizes)."""
    w = np.array([np.prod(b["n"]) * b["nlevels"] * b["ncomp"] for b in blocks], np.float64)
    cum = np.cumsum(w) / max(w.sum(), 1.0)
    owner = np.minimum((cum * world - 1e-9).astype(np.int64), world - 1)
    return [int(o) for o in np.maximum.accumulate(owner)]


def _read_boxes(s):
    """(source block, lo, hi) bounding boxes of the cells sub-matrix ``s``
    reads, one per source block."""
    kind = s["kind"]
    boxes = {}

    def add(b, cells):
        cells = np.asarray(cells, np.int64).reshape(-1, 3)
        if not len(cells):
            return
        lo, hi = cells.min(0), cells.max(0) + 1
        if b in boxes:
            lo = np.minimum(lo, boxes[b][0])
            hi = np.maximum(hi, boxes[b][1])
        boxes[b] = (lo, hi)

    if kind == specs.BC_MAP:
        lo, hi = [], []
        for d in range(3):
            pd = s["perm"][d]
            ends = [s["sign"][d] * g + s["offset"][d] for g in (s["lo"][pd], s["hi"][pd] - 1)]
            lo.append(min(ends))
            hi.append(max(ends))
        add(int(s["src_block"]), [lo, hi])
    elif kind in (specs.BC_CSR, specs.BC_SYNC):
        cb = np.asarray(s["col_block"]).reshape(-1)
        ijk = np.asarray(s["col_ijk"]).reshape(-1, 3)
        for b in np.unique(cb):
            add(int(b), ijk[cb == b])
    elif kind == specs.BC_INTERP:
        if s.get("geometry", specs.BC_GEOM_USER) != specs.BC_GEOM_USER:
            raise NotImplementedError("cubed-sphere geometry is generated on the device; "
                                      "partition user tables or CSR rows")
        sb = np.asarray(s["itp_src_block"]).reshape(-1)
        st = np.asarray(s["itp_start"]).reshape(-1, 3)
        ax = np.asarray(s["itp_axis"]).reshape(-1)
        for b in np.unique(sb):
            m = sb == b
            last = st[m].copy()
            last[np.arange(m.sum()), ax[m]] += s["p"] - 1
            add(int(b), np.concatenate([st[m], last]))
    return boxes


class Partition:
    """What rank ``rank`` of ``owner`` (one rank per block) sends, receives
    and applies.

    ``recv``: ``(peer, block, lo, hi)`` boxes this rank receives, by peer then
    block; ``send``: ``(peer, block, lo, hi)`` boxes of its own blocks it
    sends, by peer then block (the receiver's order); ``owned``: its blocks
    (global ids, ascending); ``local_blocks`` / ``local_subs``: the grid of
    the owned blocks followed by one staging block per received box, and
    the sub-matrices of the owned blocks with every remote column moved
    into its staging block."""

    def __init__(self, blocks, subs, owner, rank):
        self.rank = rank
        self.owner = list(owner)
        self._lc = [blk["nlevels"] * blk["ncomp"] for blk in blocks]
        reads = {}
        for s in subs:
            r = owner[s["block"]]
            for b, (lo, hi) in _read_boxes(s).items():
                if owner[b] == r:
                    continue
                if (r, b) in reads:
                    plo, phi = reads[(r, b)]
                    lo, hi = np.minimum(lo, plo), np.maximum(hi, phi)
                reads[(r, b)] = (lo, hi)
        box = lambda lo, hi: (tuple(int(v) for v in lo), tuple(int(v) for v in hi))  # noqa: E731
        self.recv = sorted((owner[b], b) + box(*reads[(r, b)]) for (r, b) in reads if r == rank)
        self.send = sorted((r, b) + box(*reads[(r, b)]) for (r, b) in reads if owner[b] == rank)
        self.owned = [b for b in range(len(blocks)) if owner[b] == rank]
        local = {b: i for i, b in enumerate(self.owned)}
        self.local_index = local
        stage = {b: (len(self.owned) + t, lo) for t, (_, b, lo, hi) in enumerate(self.recv)}
        self.stage_blocks = []
        for _, b, lo, hi in self.recv:
            src = blocks[b]
            self.stage_blocks.append({"n": tuple(h - l for l, h in zip(lo, hi)), "h": (0, 0, 0),
                                      "nlevels": src["nlevels"], "ncomp": src["ncomp"]})
        self.local_subs = [self._remap(s, local, stage) for s in subs
                           if owner[s["block"]] == rank]

    def _remap(self, s, local, stage):
        s = dict(s)
        s["block"] = local[s["block"]]
        kind = s["kind"]

        def where(b):
            return (local[b], np.zeros(3, np.int64)) if b in local else \
                (stage[b][0], np.asarray(stage[b][1], np.int64))
        if kind == specs.BC_MAP:
            nb, lo = where(int(s["src_block"]))
            s["src_block"] = nb
            s["offset"] = tuple(int(o - l) for o, l in zip(s["offset"], lo))
        elif kind in (specs.BC_CSR, specs.BC_SYNC):
            cb = np.asarray(s["col_block"], np.int32).reshape(-1).copy()
            ijk = np.asarray(s["col_ijk"], np.int64).reshape(-1, 3).copy()
            for b in np.unique(cb):
                m = cb == b
                nb, lo = where(int(b))
                cb[m] = nb
                ijk[m] -= lo
            s["col_block"], s["col_ijk"] = cb, ijk.astype(np.int32)
        elif kind == specs.BC_INTERP:
            sb = np.asarray(s["itp_src_block"], np.int32).reshape(-1).copy()
            st = np.asarray(s["itp_start"], np.int64).reshape(-1, 3).copy()
            for b in np.unique(sb):
                m = sb == b
                nb, lo = where(int(b))
                sb[m] = nb
                st[m] -= lo
            s["itp_src_block"], s["itp_start"] = sb, st.astype(np.int32)
        return s

    def peers(self, which):
        """``{peer: (first, count)}`` element ranges of the send or receive
        buffer per peer (boxes of one peer are consecutive)."""
        lst = self.send if which == "send" else self.recv
        out, pos = {}, 0
        for peer, b, lo, hi in lst:
            n = self.box_values(peer, b, lo, hi)
            first, cnt = out.get(peer, (pos, 0))
            out[peer] = (first, cnt + n)
            pos += n
        return out

    def box_values(self, peer, b, lo, hi):
        """Values of one box: its cells times the block's levels and
        components."""
        return int(np.prod([h - l for l, h in zip(lo, hi)])) * self._lc[b]


def transfer(send_ranges, recv_ranges, sendbuf, recvbuf, group=None):
    """Grouped point-to-point sends and receives of every peer's slice of
    the send and receive buffers (one batch, then wait)."""
    import torch.distributed as dist
    ops = []
    for peer, (a, n) in sorted(send_ranges.items()):
        ops.append(dist.P2POp(dist.isend, sendbuf[a:a + n], peer, group))
    for peer, (a, n) in sorted(recv_ranges.items()):
        ops.append(dist.P2POp(dist.irecv, recvbuf[a:a + n], peer, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class GhostExchange:
    """The ghost fill of the owned blocks of one rank: pack the boxes other
    ranks read, exchange them, apply the local plan.

    ``tensors``: the owned blocks' fields, ``(C, L, F2, F1, F0)`` per block in
    ``partition.owned`` order, on this rank's device; the plan is built for
    their strides.  :meth:`apply` runs the three steps; they are also
    callable one by one (:meth:`pack_boxes`, :meth:`transfer`,
    :meth:`local_apply`)."""

    def __init__(self, blocks, subs, dtype, owner, rank, tensors, opts=None):
        import torch
        part = Partition(blocks, subs, owner, rank)
        self.part = part
        self.dtype = dtype
        dev = tensors[0].device
        tdt = torch.float32 if dtype == "f32" else torch.float64
        own = bc.block_descriptors(tensors, [blocks[b] for b in part.owned])
        self.recvbuf = torch.empty(sum(part.box_values(*r) for r in part.recv), dtype=tdt,
                                   device=dev)
        self.staging, pos = [], 0
        for blk in part.stage_blocks:
            n = blk["n"]
            shape = (blk["ncomp"], blk["nlevels"], n[2], n[1], n[0])
            cnt = int(np.prod(shape))
            self.staging.append(self.recvbuf[pos:pos + cnt].view(shape))
            pos += cnt
        stage_desc = [specs.contiguous_block(b) for b in part.stage_blocks]
        self.pack = bc.Pack(own, [(part.local_index[b], lo, hi) for _, b, lo, hi in part.send],
                            dtype)
        self.sendbuf = torch.empty(max(self.pack.size, 1), dtype=tdt, device=dev)
        self.plan = bc.Plan(own + stage_desc, part.local_subs, dtype, opts)
        self.send_ranges = part.peers("send")
        self.recv_ranges = part.peers("recv")
        self._n_owned = len(part.owned)

    def pack_boxes(self, tensors, stream=None):
        if self.pack.size:
            self.pack.run(bc.slot_table(tensors), self.sendbuf, stream)

    def transfer(self, group=None):
        """Grouped sends and receives of every peer's boxes (one batch)."""
        transfer(self.send_ranges, self.recv_ranges, self.sendbuf, self.recvbuf, group)

    def local_apply(self, tensors, stream=None):
        fields = list(tensors) + self.staging
        self.plan.check_tensors(fields)
        self.plan.apply(bc.slot_table(fields), stream=stream)

    def apply(self, tensors, stream=None, group=None):
        """Pack, exchange, then fill every covered ghost of the owned
        blocks (in place)."""
        self.pack_boxes(tensors, stream)
        self.transfer(group)
        self.local_apply(tensors, stream)
