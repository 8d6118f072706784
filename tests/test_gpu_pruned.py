"""Dead-ghost elimination on the GPU (``bc_plan_create_pruned``, Sec. IV-C):
the live ghost values equal the oracle's rows, bit for bit on copies and
within the row-scaled tolerance elsewhere; dead ghost values and data are
untouched; the adjoint is the oracle's transpose restricted to the live
rows.  Liveness comes from the shift-based definition in ``pruning.py``."""
import numpy as np
import pytest

from gpu_util import TOL, bits, compare, flat, to_device, to_device_innermost
from oracle.operator import Operator, apply_adjoint, build_operator
from paper_2605_14780_gb300 import bc, synth
from pruning import live_mask

pytestmark = pytest.mark.gpu


def _restrict(op, live):
    keep = live[op.rows]
    return Operator(op.layout, op.rows[keep], op.A[keep], op.b[keep])


def _run(w, stencil, layout="outer", opts=None):
    import torch
    dev = to_device_innermost if layout == "inner" else to_device
    ts = dev(w["fields"])
    plan = bc.plan_for_workload(w, ts, opts, stencil=stencil)
    plan.apply(bc.slot_table(ts))
    torch.cuda.synchronize()
    return plan, [t.cpu().numpy() for t in ts]


CASES = [
    ("alg1_star", lambda: synth.alg1_example(dtype="f64"), bc.star_stencil(2, 1)),
    ("alg1_box", lambda: synth.alg1_example(dtype="f64"), bc.box_stencil(2, 1)),
    ("hpcg_P_7pt", lambda: synth.hpcg_block((9, 7, 6), "P", seed=2), bc.star_stencil(3, 1)),
    ("hpcg_S_27pt", lambda: synth.hpcg_block((9, 7, 6), "S", seed=2), bc.box_stencil(3, 1)),
    ("batching_star", lambda: synth.batching(nblocks=40, side_lo=3, side_hi=30, lev_lo=1,
                                             lev_hi=19, h=2, seed=5, dtype="f32"),
     bc.star_stencil(2, 1)),
    ("batching_box", lambda: synth.batching(nblocks=40, side_lo=3, side_hi=30, lev_lo=1,
                                            lev_hi=19, h=2, seed=6, dtype="f32"),
     bc.box_stencil(2, 1)),
    ("sphere_star2", lambda: synth.cubed_sphere(9, 3, 6, 3, ("h", "u", "v"), "f64", seed=3),
     bc.star_stencil(2, 2)),
]


@pytest.mark.parametrize("name,make,stencil", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("layout", ["outer", "inner"])
def test_pruned_forward(name, make, stencil, layout):
    w = make()
    live = live_mask(w, stencil)
    plan, out = _run(w, stencil, layout)
    op = _restrict(build_operator(w), live)
    compare(w, out, op=op)
    # the plan holds exactly the live ghost values that some sub-matrix covers
    assert plan.stats()["ghost_values"] == len(op.rows)


def test_pruned_with_the_full_stencil_equals_the_plan():
    """A 27-point stencil reads every ghost of an h = 1 frame: the pruned plan
    writes the same bits as the unpruned one."""
    import torch
    w = synth.hpcg_block((8, 6, 5), "S", seed=4)
    _, a = _run(w, bc.box_stencil(3, 1))
    ts = to_device(w["fields"])
    bc.plan_for_workload(w, ts).apply(bc.slot_table(ts))
    torch.cuda.synchronize()
    assert np.array_equal(bits(flat(a)), bits(flat([t.cpu().numpy() for t in ts])))


@pytest.mark.parametrize("name,make,stencil", CASES[2:], ids=[c[0] for c in CASES[2:]])
def test_pruned_adjoint(name, make, stencil):
    import torch
    w = make()
    live = live_mask(w, stencil)
    ts = to_device(w["fields"])
    plan = bc.plan_for_workload(w, ts, stencil=stencil)
    cot = synth.cotangent_like(w, 31)
    cs = to_device(cot)
    plan.adjoint(bc.slot_table(cs))
    torch.cuda.synchronize()
    op = _restrict(build_operator(w), live)
    ref = flat(apply_adjoint(op, cot))
    got = flat([c.cpu().numpy() for c in cs]).astype(np.float64)
    y = flat(cot).astype(np.float64)
    covered = np.zeros(y.size, bool)
    covered[op.rows] = True
    assert np.all(got[covered] == 0.0)
    # dead ghosts (and uncovered values) keep their cotangent bit for bit
    untouched = ~covered
    dr = op.layout.data_rows()
    touched = np.zeros(y.size, bool)
    touched[dr[np.unique(op.A.indices)]] = True
    same = untouched & ~touched
    assert np.array_equal(bits(flat([c.cpu().numpy() for c in cs]))[same], bits(flat(cot))[same])
    scale = np.abs(y).copy()
    scale[dr] += abs(op.A).T @ np.abs(y[op.rows])
    tol = TOL[w["dtype"]]
    err = np.abs(got[touched] - ref[touched])
    assert np.all(err <= tol * scale[touched])


def test_pruned_strict_cover_and_empty_stencil():
    import torch
    w = synth.batching(nblocks=12, side_lo=4, side_hi=20, lev_lo=1, lev_hi=5, h=2,
                       seed=9, dtype="f32")
    ts = to_device(w["fields"])
    # every live ghost is covered: strict mode accepts the pruned plan
    bc.plan_for_workload(w, ts, {"strict_cover": 1}, stencil=bc.star_stencil(2, 1))
    with pytest.raises(bc.BCError) as e:
        bc.plan_for_workload(w, ts, stencil=np.zeros((0, 3), np.int32))
    assert e.value.status == "BC_ERR_INVALID_ARG"
    torch.cuda.synchronize()


def test_pruned_batching_512_star_sampled():
    """The 512-block workload pruned for a 5-point stencil: half the ghost
    layers and the corners are dead."""
    w = synth.batching()
    stencil = bc.star_stencil(2, 1)
    live = live_mask(w, stencil)
    plan, out = _run(w, stencil, "inner")
    op = _restrict(build_operator(w), live)
    compare(w, out, op=op)
    assert plan.stats()["ghost_values"] == len(op.rows)
