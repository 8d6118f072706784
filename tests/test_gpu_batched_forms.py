"""The two executions of the batched forward -- the persistent work-list
launch and one kernel per family -- with 16-byte vector runs and with scalar
runs, at every level-chunk split, on fields whose slot pointers are not
16-byte aligned: bit-identical to each other and to the oracle (copies and
zero rows), and the adjoint's vector add-runs bit-identical to the scalar
ones."""
import numpy as np
import pytest

from gpu_util import bits, compare, flat
from oracle.operator import apply_adjoint, build_operator
from paper_2605_14780_gb300 import bc, synth

pytestmark = pytest.mark.gpu

P, F, FP = bc.BC_BATCH_PERSISTENT, bc.BC_BATCH_FAMILIES, bc.BC_BATCH_FAMILIES_PERSISTENT
S1 = bc.BC_BATCH_SINGLE


def _packed(arrays, shift, layout):
    """One device buffer holding the blocks back to back after `shift`
    leading elements, so that slot pointers fall on every alignment; views
    in (C, L, F2, F1, F0) index order."""
    import torch
    total = shift + sum(a.size for a in arrays)
    dt = torch.from_numpy(arrays[0][:0]).dtype
    buf = torch.zeros(total, dtype=dt, device="cuda")
    views, pos = [], shift
    for a in arrays:
        C, L, F2, F1, F0 = a.shape
        if layout == "innermost":
            v = buf[pos:pos + a.size].view(C, F2, F1, F0, L).permute(0, 4, 1, 2, 3)
        else:
            v = buf[pos:pos + a.size].view(a.shape)
        v.copy_(torch.from_numpy(a))
        views.append(v)
        pos += a.size
    return buf, views


def _forward(w, opts, shift, layout):
    import torch
    _, ts = _packed(w["fields"], shift, layout)
    plan = bc.plan_for_workload(w, ts, opts)
    table = bc.slot_table(ts)
    for _ in range(3):  # repeated launches: the work counter resets itself
        plan.apply(table)
    torch.cuda.synchronize()
    return plan, [t.cpu().numpy() for t in ts]


def _adjoint(w, plan, cot, shift, layout):
    import torch
    _, cs = _packed(cot, shift, layout)
    plan.adjoint(bc.slot_table(cs))
    torch.cuda.synchronize()
    return [c.cpu().numpy() for c in cs]


OPTS = [{"batch_mode": P}, {"batch_mode": P, "scalar_runs": 1},
        {"batch_mode": F}, {"batch_mode": F, "scalar_runs": 1},
        {"batch_mode": FP}, {"batch_mode": FP, "threads": 256},
        {"batch_mode": S1}, {"batch_mode": S1, "threads": 64},
        {"batch_mode": P, "threads": 256, "units_per_lane": 8},
        {"batch_mode": P, "units_per_lane": 1, "ctas_per_sm": 1}]


@pytest.mark.parametrize("layout", ["outermost", "innermost"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("shift", [0, 1, 2, 3])
def test_vector_runs_on_every_alignment(layout, dtype, shift):
    w = synth.batching(nblocks=40, side_lo=3, side_hi=48, lev_lo=1, lev_hi=23,
                       h=2, seed=31 + shift, dtype=dtype)
    op = build_operator(w)
    cot = synth.cotangent_like(w, 32)
    ref_adj = flat(apply_adjoint(op, cot))
    outs, adjs = [], []
    for opts in OPTS:
        plan, out = _forward(w, opts, shift, layout)
        compare(w, out, op=op)
        outs.append(bits(flat(out)))
        adjs.append(flat(_adjoint(w, plan, cot, shift, layout)))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    for a in adjs[1:]:
        assert np.array_equal(bits(a), bits(adjs[0]))
    y = flat(cot).astype(np.float64)
    scale = np.abs(y).copy()
    scale[op.layout.data_rows()] += abs(op.A).T @ np.abs(y[op.rows])
    tol = 1e-12 if dtype == "f64" else 2e-6
    assert np.all(np.abs(adjs[0].astype(np.float64) - ref_adj) <= tol * scale)


@pytest.mark.parametrize("chunk", [1, 2, 4, 8])
@pytest.mark.parametrize("mode", [P, F, FP, S1])
def test_level_chunks(chunk, mode):
    """Every levels-per-lane split of the chunked unit order (levels
    outermost: interpolation with rotation, CSR corners, and the transpose
    gather): forward against the oracle, adjoint bit-identical to the
    default split (each data value sums its entries in the same order)."""
    w = synth.cubed_sphere(12, 3, 6, 11, ("h", "u", "v"), "f32", seed=33)
    opts = {"batch_mode": mode, "level_chunk": chunk}
    plan, out = _forward(w, opts, 1, "outermost")
    op = build_operator(w)
    compare(w, out, op=op)
    cot = synth.cotangent_like(w, 34)
    adj = flat(_adjoint(w, plan, cot, 1, "outermost"))
    plan0, _ = _forward(w, {}, 1, "outermost")
    adj0 = flat(_adjoint(w, plan0, cot, 1, "outermost"))
    assert np.array_equal(bits(adj), bits(adj0))


@pytest.mark.parametrize("threads", [64, 512])
@pytest.mark.parametrize("mode", [F, FP, S1])
@pytest.mark.parametrize("vector", [False, True])
def test_staged_tiles_match_per_lane_rows(threads, mode, vector):
    """Staged tiles (levels outermost: a warp's box of source values, or of
    ghost cotangents, copied to shared memory) against the per-lane rows:
    reconstruction-and-quadrature CSR rows and their transpose, or panel-edge
    interpolation with rotation; forward and adjoint bit-identical (the same
    sums in the same order) and the forward against the oracle.  512 threads
    ask for 64 KB of dynamic shared memory in the CSR kernels."""
    if vector:
        w = synth.cubed_sphere(24, 3, 6, 9, ("h", "u", "v"), "f32", seed=41)
    else:
        w = synth.cubed_sphere(24, 3, 4, 9, ("h", "u", "v"), "f32", seed=41, quad=2)
    cot = synth.cotangent_like(w, 42)
    res = []
    for unstaged in (0, 1):
        opts = {"batch_mode": mode, "threads": threads, "unstaged_rows": unstaged}
        plan, out = _forward(w, opts, 1, "outermost")
        adj = _adjoint(w, plan, cot, 1, "outermost")
        res.append((plan.stats()["nitems"], flat(out), flat(adj)))
    assert res[0][0] != res[1][0]  # the default plan does stage some tiles
    assert np.array_equal(bits(res[0][1]), bits(res[1][1]))
    assert np.array_equal(bits(res[0][2]), bits(res[1][2]))
    _, out = _forward(w, {"batch_mode": mode, "threads": threads}, 1, "outermost")
    compare(w, out, op=build_operator(w))


@pytest.mark.parametrize("mode", [P, FP])
def test_persistent_launches_on_several_streams(mode):
    """Applies of one persistent plan alternating over three streams (one
    work counter each) and a captured graph replayed on another stream,
    every result against the oracle."""
    import torch
    w = synth.batching(nblocks=64, side_lo=4, side_hi=64, lev_lo=1, lev_hi=40,
                       h=2, seed=35, dtype="f32")
    op = build_operator(w)
    sets = [_packed(w["fields"], k, "innermost") for k in range(3)]
    plan = bc.plan_for_workload(w, sets[0][1], {"batch_mode": mode})
    streams = [torch.cuda.Stream() for _ in range(3)]
    tables = [bc.slot_table(v) for _, v in sets]
    for rep in range(4):
        for k in range(3):
            plan.apply(tables[k], stream=streams[(k + rep) % 3])
    torch.cuda.synchronize()
    for _, v in sets:
        compare(w, [t.cpu().numpy() for t in v], op=op)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=s):
        plan.apply(tables[0], stream=s)
    for t, a in zip(sets[0][1], w["fields"]):
        t.copy_(torch.from_numpy(a))
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    compare(w, [t.cpu().numpy() for t in sets[0][1]], op=op)


def test_stats_count_one_launch_for_the_persistent_form():
    w = synth.batching(nblocks=20, side_lo=4, side_hi=30, lev_lo=1, lev_hi=9,
                       h=2, seed=36, dtype="f32")
    _, ts = _packed(w["fields"], 0, "innermost")
    assert bc.plan_for_workload(w, ts, {"batch_mode": P}).stats()["launches_fwd"] == 1
    assert bc.plan_for_workload(w, ts, {"batch_mode": F}).stats()["launches_fwd"] == 2
    assert bc.plan_for_workload(w, ts, {"batch_mode": FP}).stats()["launches_fwd"] == 2
    assert bc.plan_for_workload(w, ts, {"batch_mode": S1}).stats()["launches_fwd"] == 1


def test_autotune_result_cache(tmp_path, monkeypatch):
    """bc_plan_autotune stores its choice under the plan's hash in
    BC_AUTOTUNE_CACHE; a second plan of the same operator and layout takes
    the stored options without timing (no new line), and both still give the
    oracle's ghosts.  A plan of another layout gets its own line."""
    import torch
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("BC_AUTOTUNE_CACHE", str(path))
    w = synth.batching(nblocks=30, side_lo=4, side_hi=40, lev_lo=1, lev_hi=20,
                       h=2, seed=37, dtype="f32")
    op = build_operator(w)
    _, ts = _packed(w["fields"], 1, "innermost")
    plan = bc.plan_for_workload(w, ts)
    plan.autotune(bc.slot_table(ts))
    lines = path.read_text().splitlines()
    assert len(lines) == 1
    tuned = plan.stats()
    _, ts2 = _packed(w["fields"], 1, "innermost")
    plan2 = bc.plan_for_workload(w, ts2)
    plan2.autotune(bc.slot_table(ts2))
    assert path.read_text().splitlines() == lines
    st2 = plan2.stats()
    for k in ("form_threads", "form_ctas_per_sm", "units_per_lane", "launches_fwd"):
        assert st2[k] == tuned[k], k
    for t, a in zip(ts2, w["fields"]):
        t.copy_(torch.from_numpy(a))
    plan2.apply(bc.slot_table(ts2))
    torch.cuda.synchronize()
    compare(w, [t.cpu().numpy() for t in ts2], op=op)
    _, ts3 = _packed(w["fields"], 1, "outermost")
    bc.plan_for_workload(w, ts3).autotune(bc.slot_table(ts3))
    assert len(path.read_text().splitlines()) == 2
