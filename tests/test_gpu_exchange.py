"""The distributed ghost exchange's GPU path on one GPU: two ranks' parts
in one process -- each packs the boxes its peer reads with the library's
pack kernel, the buffers are handed over by device copies (what the grouped
sends and receives do between GPUs), then each applies its local plan
(owned blocks plus the received boxes).  No kernel waits on another rank.
Every owned ghost against the single-process oracle (copies bit for bit)."""
import numpy as np
import pytest

from gpu_util import compare, to_device, to_device_innermost
from paper_2605_14780_gb300 import bc, exchange, specs, synth

pytestmark = pytest.mark.gpu


def _run_two_ranks(w, layout="outermost"):
    import torch
    subs = specs.submatrices(w)
    nb = len(w["blocks"])
    owner = [b % 2 for b in range(nb)]
    dev = to_device_innermost if layout == "innermost" else to_device
    fields = dev(w["fields"])
    exs, owned = [], []
    for r in range(2):
        mine = [fields[b] for b in range(nb) if owner[b] == r]
        owned.append(mine)
        exs.append(exchange.GhostExchange(w["blocks"], subs, w["dtype"], owner, r, mine))
    for ex, mine in zip(exs, owned):
        ex.pack_boxes(mine)
    for r in range(2):
        for peer, (a, n) in exs[r].recv_ranges.items():
            a2, n2 = exs[peer].send_ranges[r]
            assert n == n2
            exs[r].recvbuf[a:a + n].copy_(exs[peer].sendbuf[a2:a2 + n2])
    for ex, mine in zip(exs, owned):
        ex.local_apply(mine)
    torch.cuda.synchronize()
    return exs, [f.cpu().numpy() for f in fields]


@pytest.mark.parametrize("layout", ["outermost", "innermost"])
@pytest.mark.parametrize("make", [
    lambda: synth.batching(nblocks=24, side_lo=8, side_hi=9, lev_lo=3, lev_hi=3, h=2, seed=53,
                           dtype="f32"),
    lambda: synth.batching(nblocks=40, side_lo=3, side_hi=30, lev_lo=1, lev_hi=12, h=2,
                           seed=54, dtype="f64"),
    lambda: synth.staggered_interp(nlevels=4, p=4, dtype="f64"),
    lambda: synth.two_level(20, 14, 2, nlevels=3, ncomp=2, dtype="f32", seed=55),
])
def test_two_ranks_match_one_process(make, layout):
    w = make()
    exs, out = _run_two_ranks(w, layout)
    compare(w, out)
    assert sum(len(ex.part.recv) for ex in exs) > 0


def test_pack_kernel_layout():
    """bc_pack_run stores each box [component][level][k][j][i], boxes back
    to back, bit for bit."""
    import torch
    w = synth.batching(nblocks=6, side_lo=5, side_hi=12, lev_lo=2, lev_hi=5, h=2, seed=56,
                       dtype="f32")
    ts = to_device_innermost(w["fields"])
    descs = bc.block_descriptors(ts, w["blocks"])
    boxes = [(0, (-2, 0, 0), (3, 4, 1)), (3, (1, -1, 0), (4, 2, 1)), (5, (0, 0, 0), (1, 1, 1))]
    pk = bc.Pack(descs, boxes, "f32")
    buf = torch.empty(pk.size, dtype=torch.float32, device="cuda")
    pk.run(bc.slot_table(ts), buf)
    torch.cuda.synchronize()
    want = []
    for b, lo, hi in boxes:
        h = w["blocks"][b]["h"]
        a = w["fields"][b]
        want.append(a[:, :, lo[2] + h[2]:hi[2] + h[2], lo[1] + h[1]:hi[1] + h[1],
                      lo[0] + h[0]:hi[0] + h[0]].ravel())
    want = np.concatenate(want)
    assert np.array_equal(buf.cpu().numpy().view(np.uint32), want.view(np.uint32))
    with pytest.raises(bc.BCError) as e:
        bc.Pack(descs, [(0, (-3, 0, 0), (1, 1, 1))], "f32")
    assert e.value.status == "BC_ERR_OUT_OF_RANGE"
