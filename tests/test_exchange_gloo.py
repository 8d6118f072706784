"""Distributed ghost exchange (Sec. V-B bounding boxes) on CPU ranks over
gloo: every rank plans its boxes, packs what its peers read (the layout of
bc_pack_run, emulated on the host), exchanges them with the library's
grouped point-to-point transfer, and evaluates the rows of its local plan
(owned blocks plus the received boxes, from a host-only plan's exported
rows).  The owned ghosts must equal the single-process oracle's: bit for
bit on copy and zero rows, within 1e-13 of the row scale elsewhere."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _workload(name):
    from paper_2605_14780_gb300 import synth
    if name == "batching":
        # equal edge lengths and level counts: many halo copies between blocks
        return synth.batching(nblocks=14, side_lo=8, side_hi=9, lev_lo=3, lev_hi=3, h=2,
                              seed=51, dtype="f32")
    if name == "staggered":
        return synth.staggered_interp(nlevels=3, p=4, dtype="f64")
    if name == "two_level":
        return synth.two_level(20, 14, 2, nlevels=3, ncomp=2, dtype="f64", seed=52)
    raise ValueError(name)


def _worker(rank, world, port, name, out):
    import torch
    import torch.distributed as dist
    from exchange_util import apply_rows, local_descs, pack_host, staging_views
    from oracle.operator import apply, build_operator, row_scale
    from paper_2605_14780_gb300 import bc, exchange, specs
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _workload(name)
        subs = specs.submatrices(w)
        # blocks dealt out in turn, so that most halo reads cross ranks
        owner = [b % world for b in range(len(w["blocks"]))]
        part = exchange.Partition(w["blocks"], subs, owner, rank)
        send = torch.from_numpy(pack_host(w["fields"], w["blocks"], part.send).copy())
        recv = torch.empty(sum(part.box_values(*r) for r in part.recv), dtype=send.dtype)
        exchange.transfer(part.peers("send"), part.peers("recv"), send, recv)
        local = [w["fields"][b].copy() for b in part.owned] + \
            staging_views(recv.numpy(), part.stage_blocks)
        descs = local_descs(w, part)
        plan = bc.Plan(descs, part.local_subs, w["dtype"], {"host_only": 1})
        got = apply_rows(plan.export_csr(), local, descs)
        # the single-process oracle, on the owned blocks' ghosts
        op = build_operator(w)
        ref = op.layout.flatten_full(apply(op, w["fields"]))
        scale = np.zeros(ref.size)
        scale[op.rows] = row_scale(op, w["fields"])
        covered = np.zeros(ref.size, bool)
        covered[op.rows] = True
        nrows = op.A.indptr
        unit = np.zeros(ref.size, bool)
        one = (np.diff(nrows) == 1) & (op.b == 0)
        one[one] = op.A.data[nrows[:-1][one]] == 1.0
        unit[op.rows[one | (np.diff(nrows) == 0)]] = True
        slot_base, k = [], 0
        for lb, b in enumerate(part.owned):
            slot_base.append(k)
            k += w["blocks"][b]["ncomp"]
        checked = 0
        sizes = [a.size for a in w["fields"]]
        starts = np.concatenate([[0], np.cumsum(sizes)])
        for lb, b in enumerate(part.owned):
            C = w["blocks"][b]["ncomp"]
            per = sizes[b] // C
            for c in range(C):
                for e in range(per):
                    g = starts[b] + c * per + e
                    if not covered[g]:
                        continue
                    v = got[(slot_base[lb] + c, e)]
                    if unit[g]:
                        dt = w["fields"][0].dtype
                        assert np.asarray(v, dt).view(np.uint64 if dt == np.float64 else np.uint32) \
                            == np.asarray(ref[g], dt).view(np.uint64 if dt == np.float64 else np.uint32)
                    else:
                        assert abs(v - ref[g]) <= 1e-13 * scale[g]
                    checked += 1
        out[rank] = (checked, len(part.recv), len(part.send))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["batching", "staggered", "two_level"])
def test_exchange_then_local_apply_matches_the_oracle(name):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = dict(out)
    assert set(res) == {0, 1}
    assert sum(r[0] for r in res.values()) > 0
    # remote reads happened, and every box received was sent
    assert sum(r[1] for r in res.values()) > 0
    assert sum(r[1] for r in res.values()) == sum(r[2] for r in res.values())


def test_partition_boxes_are_bounding_boxes():
    """Host planning only: the received boxes cover exactly the remote
    cells the owned rows read (bounding box: every read inside, every face
    of the box touched), and sender and receiver agree on the boxes."""
    from paper_2605_14780_gb300 import exchange, specs, synth
    w = synth.batching(nblocks=14, side_lo=4, side_hi=24, lev_lo=1, lev_hi=6, h=2,
                       seed=51, dtype="f32")
    subs = specs.submatrices(w)
    owner = exchange.owners_by_cells(w["blocks"], 3)
    parts = [exchange.Partition(w["blocks"], subs, owner, r) for r in range(3)]
    for r, p in enumerate(parts):
        for peer, b, lo, hi in p.recv:
            assert (r, b, lo, hi) in [(x[0], x[1], x[2], x[3]) for x in parts[peer].send]
            # the owned rows' reads of block b, from the oracle's row sets
            cells = []
            for s in subs:
                if owner[s["block"]] != r:
                    continue
                for bb, (blo, bhi) in exchange._read_boxes(s).items():
                    if bb == b:
                        cells += [blo, bhi - 1]
            cells = np.array(cells)
            assert tuple(cells.min(0)) == lo and tuple(cells.max(0) + 1) == hi
