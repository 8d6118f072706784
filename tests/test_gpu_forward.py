"""GPU parity of the forward apply against the FP64 oracle, through the C ABI.

Copies, zero and constant rows bit-exact; interpolation and CSR rows within
1e-12 (FP64) / 2e-6 (FP32) of the row scale sum_e |a_ie x_e| + |b_i|.
"""
import numpy as np
import pytest

from gpu_util import bits, compare, flat, run, to_device, to_device_innermost
from oracle.operator import build_operator
from paper_2605_14780_gb300 import bc, synth

pytestmark = pytest.mark.gpu

FORMS = [bc.BC_FORM_BATCHED, bc.BC_FORM_TYPEWIDE, bc.BC_FORM_PER_BC]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_alg1(dtype):
    w = synth.alg1_example(dtype=dtype)
    _, out = run(w)
    compare(w, out)


@pytest.mark.parametrize("variant", ["Z", "P", "S"])
@pytest.mark.parametrize("n", [(6, 6, 6), (9, 7, 5), (1, 1, 1)])
def test_hpcg_small(variant, n):
    w = synth.hpcg_block(n, variant, seed=4)
    _, out = run(w)
    compare(w, out)


@pytest.mark.parametrize("variant", ["Z", "P", "S"])
def test_hpcg_128_full(variant):
    """The 128^3 HPCG-like block, checked in full and through the 27-point
    operator applied to the ghost-filled array."""
    from oracle.operator import apply
    w = synth.hpcg_block(128, variant, seed=2)
    _, out = run(w)
    op, nexact, _ = compare(w, out)
    assert nexact == len(op.rows) == 130 ** 3 - 128 ** 3
    # the 27-point operator (diagonal 26, off-diagonals -1) on the GPU's and
    # on the oracle's ghost-filled arrays
    ref = apply(op, w["fields"])

    def stencil27(full):
        x = full[0, 0]
        box = np.zeros((128, 128, 128))
        for dk in range(3):
            for dj in range(3):
                for di in range(3):
                    box += x[dk:dk + 128, dj:dj + 128, di:di + 128]
        return 27.0 * x[1:-1, 1:-1, 1:-1] - box
    assert np.array_equal(stencil27(out[0].astype(np.float64)), stencil27(ref[0]))


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("seed", [1, 2])
def test_batching_small(dtype, seed):
    w = synth.batching(nblocks=48, side_lo=3, side_hi=40, lev_lo=1, lev_hi=19,
                       h=2, seed=seed, dtype=dtype)
    _, out = run(w)
    compare(w, out)


@pytest.mark.parametrize("form", FORMS)
def test_forms_bit_identical(form):
    w = synth.batching(nblocks=64, side_lo=4, side_hi=64, lev_lo=1, lev_hi=40,
                       h=2, seed=7, dtype="f32")
    _, ref = run(w, bc.BC_FORM_BATCHED)
    _, out = run(w, form)
    assert np.array_equal(bits(flat(out)), bits(flat(ref)))
    compare(w, out)


@pytest.mark.parametrize("opts", [
    {"ctas_per_sm": 2, "threads": 128, "units_per_lane": 1},
    {"ctas_per_sm": 4, "threads": 256, "units_per_lane": 8},
    {"ctas_per_sm": 1, "threads": 512, "units_per_lane": 3},
    {"ctas_per_sm": 0, "threads": 128, "units_per_lane": 64},
])
def test_persistent_and_item_shapes(opts):
    """The persistent work-list launch (warps claim items from a device
    counter) with several resident-grid sizes, repeated launches (the
    counter must reset itself), odd item shapes."""
    w = synth.batching(nblocks=64, side_lo=4, side_hi=64, lev_lo=1, lev_hi=40,
                       h=2, seed=8, dtype="f32")
    _, out = run(w, opts=opts, repeat=3)
    compare(w, out)


@pytest.mark.parametrize("make", [
    lambda: synth.hpcg_block((1, 1, 1), "P", seed=3),
    lambda: synth.hpcg_block((1, 1, 1), "S", seed=3, dtype="f32"),
    lambda: synth.hpcg_block((2, 1, 3), "P", seed=3),
    lambda: synth.batching(nblocks=6, side_lo=1, side_hi=3, lev_lo=1, lev_hi=3, h=1, seed=5,
                           dtype="f32"),
])
def test_degenerate_block_sizes(make):
    """One-cell extents (h = N = 1 reflections, one-cell blocks): forward
    bit-exact against the oracle, and the adjoint."""
    import torch
    from oracle.operator import apply_adjoint
    w = make()
    plan, out = run(w)
    compare(w, out)
    cot = synth.cotangent_like(w, 9)
    cs = to_device(cot)
    plan.adjoint(bc.slot_table(cs))
    torch.cuda.synchronize()
    got = flat([c.cpu().numpy() for c in cs]).astype(np.float64)
    op = build_operator(w)
    ref = flat(apply_adjoint(op, cot))
    y = flat(cot).astype(np.float64)
    scale = np.abs(y).copy()
    scale[op.layout.data_rows()] += abs(op.A).T @ np.abs(y[op.rows])
    tol = 1e-12 if w["dtype"] == "f64" else 2e-6
    assert np.all(np.abs(got - ref) <= tol * scale)


@pytest.mark.parametrize("unit_order", [1, 2])
@pytest.mark.parametrize("layout", ["outermost", "innermost"])
def test_forced_unit_orders(unit_order, layout):
    """bc_plan_opts.unit_order forces cells-fastest or levels-fastest units
    whatever the layout (the other order than the automatic one for one of
    the two layouts): forward bit-exact, adjoint within tolerance."""
    import torch
    from oracle.operator import apply_adjoint
    w = synth.batching(nblocks=24, side_lo=2, side_hi=30, lev_lo=1, lev_hi=17, h=2, seed=29,
                       dtype="f32")
    dev = to_device_innermost if layout == "innermost" else to_device
    ts = dev(w["fields"])
    plan, _ = run(w, opts={"unit_order": unit_order}, tensors=ts)
    compare(w, [t.cpu().numpy() for t in ts])
    cot = synth.cotangent_like(w, 30)
    cs = dev(cot)
    plan.adjoint(bc.slot_table(cs))
    torch.cuda.synchronize()
    got = flat([c.cpu().numpy() for c in cs]).astype(np.float64)
    op = build_operator(w)
    ref = flat(apply_adjoint(op, cot))
    y = flat(cot).astype(np.float64)
    scale = np.abs(y).copy()
    scale[op.layout.data_rows()] += abs(op.A).T @ np.abs(y[op.rows])
    assert np.all(np.abs(got - ref) <= 2e-6 * scale)


@pytest.mark.parametrize("make", [
    lambda: synth.tiny_cubed_sphere(),
    lambda: synth.cubed_sphere(9, 3, 6, 5, ("h", "u", "v"), "f32", seed=4),
    lambda: synth.batching(nblocks=20, side_lo=2, side_hi=30, lev_lo=1, lev_hi=9, h=2, seed=8,
                           dtype="f32"),
])
def test_work_replay_of_device_plans(make):
    """The host replay of the work lists on plans built with the GPU
    geometry (interpolation tables generated on the device)."""
    w = make()
    plan = bc.plan_for_workload(w, to_device(w["fields"]))
    n, bad, msg = plan.check_work()
    assert n > 0 and bad == 0, msg


def test_no_adjoint_plans_refuse_the_adjoint():
    w = synth.alg1_example()
    ts = to_device(w["fields"])
    plan = bc.plan_for_workload(w, ts, {"no_adjoint": 1})
    with pytest.raises(bc.BCError) as e:
        plan.adjoint(bc.slot_table(ts))
    assert e.value.status == "BC_ERR_UNSUPPORTED"


def test_batching_full_512():
    """The 512-block batching workload in full."""
    w = synth.batching()
    _, out = run(w)
    compare(w, out)


def test_batching_full_512_bench_configuration():
    """The 512-block workload as the bench times it: levels innermost,
    default plan options, the batched apply captured in a CUDA graph on a
    side stream and replayed; every ghost value against the oracle."""
    import torch
    w = synth.batching()
    ts = to_device_innermost(w["fields"])
    plan = bc.plan_for_workload(w, ts)
    table = bc.slot_table(ts)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.apply(table, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.apply(table, stream=s)
    for t, a in zip(ts, w["fields"]):
        t.copy_(torch.from_numpy(a))         # back to the input, ghosts NaN
    g.replay()
    torch.cuda.synchronize()
    compare(w, [t.cpu().numpy() for t in ts])


@pytest.mark.parametrize("N,h,p", [(5, 2, 4), (8, 3, 6), (16, 2, 4), (7, 1, 2),
                                   (9, 3, 8)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_cubed_sphere_scalar(N, h, p, dtype):
    w = synth.cubed_sphere(N, h, p, 3, ("scalar",), dtype, seed=N)
    _, out = run(w)
    compare(w, out)


@pytest.mark.parametrize("N,L", [(6, 1), (12, 9), (24, 8), (10, 17)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_cubed_sphere_vector(N, L, dtype):
    w = synth.cubed_sphere(N, 3, 6, L, ("h", "u", "v"), dtype, seed=3)
    _, out = run(w)
    compare(w, out)


@pytest.mark.parametrize("N,h,p,nq,fields", [(6, 2, 4, 2, ("h", "u", "v")), (9, 3, 3, 1, ("scalar",)),
                                              (10, 3, 6, 3, ("h", "u", "v")),
                                              (12, 2, 8, 4, ("scalar",)), (7, 1, 2, 5, ("h", "u", "v"))])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["outermost", "innermost"])
def test_cubed_sphere_quadrature(N, h, p, nq, fields, dtype, layout):
    """Reconstruction-and-quadrature edge rows (user CSR rows of p^2 and
    2 p^2 entries, built on the host) against the oracle."""
    from gpu_util import to_device_innermost
    w = synth.cubed_sphere(N, h, p, 5, fields, dtype, seed=N + p, quad=nq)
    ts = to_device_innermost(w["fields"]) if layout == "innermost" else None
    _, out = run(w, tensors=ts)
    compare(w, out)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["outermost", "innermost"])
def test_cubed_sphere_centred_quadrature_folded(dtype, layout):
    """Centred reconstruction patches that read the neighbour's ghosts,
    folded by 10 Jacobi sweeps at plan creation (rows of a few hundred
    entries), against the oracle."""
    from gpu_util import to_device_innermost
    w = synth.cubed_sphere(10, 3, 4, 4, ("h", "u", "v"), dtype, seed=7, quad=2, centred=True,
                           sweeps=10)
    ts = to_device_innermost(w["fields"]) if layout == "innermost" else None
    _, out = run(w, tensors=ts)
    compare(w, out)


@pytest.mark.parametrize("p,rotate", [(4, True), (2, False), (6, True), (8, False)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["outermost", "innermost"])
def test_user_interpolation_tables(p, rotate, dtype, layout):
    """Interpolation rows given as user tables (staggered neighbours, a
    per-cell rotation of the (u, v) pair) through the interpolation kernels."""
    from gpu_util import to_device_innermost
    w = synth.staggered_interp(nx=18, ny=13, h=2, nlevels=6, p=p, dtype=dtype, rotate=rotate)
    if p == 6:
        w = synth.swap_xy(w)          # stencils stepping along axis 0
    ts = to_device_innermost(w["fields"]) if layout == "innermost" else None
    _, out = run(w, tensors=ts)
    compare(w, out)


def test_hope_cubed_sphere_sampled():
    """6 x 384^2, h = 3, (h, u, v) x 32 levels FP32, 4 x 4 reconstruction at
    2 x 2 Gauss points: levels 0, 17 and 31 compared with the oracle."""
    w = synth.hope_cubed_sphere()
    _, out = run(w)
    compare(w, out, levels=[0, 17, 31])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["outermost", "innermost"])
def test_pure_function_boundary_evaluated_on_the_device(dtype, layout):
    """b = udf(i, t) written into the plan's constant tables by device code
    between graph replays of one captured apply; every step against the
    oracle's constant rows at that time, bit-exact."""
    import torch
    w = synth.dirichlet_block(dtype=dtype, t=0.0)
    ts = to_device_innermost(w["fields"]) if layout == "innermost" else to_device(w["fields"])
    plan = bc.plan_for_workload(w, ts)
    table = bc.slot_table(ts)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan.apply(table, stream=stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        plan.apply(table, stream=stream)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    for t in (1.0, 2.5, -3.0):
        with torch.cuda.stream(stream):
            for k, d in enumerate(w["bcs"]):
                jj, ii = torch.meshgrid(torch.arange(d["lo"][1], d["hi"][1], device="cuda"),
                                        torch.arange(d["lo"][0], d["hi"][0], device="cuda"),
                                        indexing="ij")
                i, j = ii.reshape(-1).double(), jj.reshape(-1).double()
                vals = torch.cat([synth.dirichlet_udf(i, j, c, t) for c in d["comps"]])
                vals = vals.to(tdt).contiguous()
                plan.set_const(k, vals, stream=stream)
                stream.synchronize()   # vals is a temporary of this loop
            g.replay()
        torch.cuda.synchronize()
        compare(synth.dirichlet_block(dtype=dtype, t=t), [x.cpu().numpy() for x in ts])


@pytest.mark.parametrize("scheme,k", [("extrapolate", 3), ("extrapolate", 1), ("smooth", 6)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["outermost", "innermost"])
def test_ghost_reading_rows_folded(scheme, k, dtype, layout):
    """User CSR rows that read other ghosts, folded by k Jacobi sweeps at
    plan creation, against the oracle's folded matrix."""
    import torch
    w = synth.ghost_on_ghost(scheme=scheme, sweeps=k, dtype=dtype, nlevels=3)
    ts = to_device_innermost(w["fields"]) if layout == "innermost" else to_device(w["fields"])
    run(w, tensors=ts)
    torch.cuda.synchronize()
    compare(w, [t.cpu().numpy() for t in ts])


def test_const_table_view():
    """The constant table as a torch view (CUDA array interface): a write
    through it is the b of the next apply."""
    import torch
    w = synth.dirichlet_block(dtype="f32", t=0.0)
    ts = to_device(w["fields"])
    plan = bc.plan_for_workload(w, ts)
    try:
        views = [plan.const_values(k) for k in range(len(w["bcs"]))]
    except (TypeError, RuntimeError) as e:
        pytest.skip(f"this torch does not import CUDA array interface views: {e}")
    wt = synth.dirichlet_block(dtype="f32", t=4.0)
    for v, d in zip(views, wt["bcs"]):
        v.copy_(torch.from_numpy(d["values"].astype(np.float32)).cuda())
    plan.apply(bc.slot_table(ts))
    torch.cuda.synchronize()
    compare(wt, [x.cpu().numpy() for x in ts])


def test_const_values_errors():
    w = synth.dirichlet_block()
    plan = bc.plan_for_workload(w, to_device(w["fields"]))
    for bad in (-1, len(w["bcs"])):
        with pytest.raises(bc.BCError) as e:
            plan.const_values(bad)
        assert e.value.status == "BC_ERR_INVALID_ARG"
    a = synth.alg1_example()
    with pytest.raises(bc.BCError) as e:
        bc.plan_for_workload(a, to_device(a["fields"])).const_values(0)
    assert e.value.status == "BC_ERR_INVALID_ARG"          # not a constant
    with pytest.raises(bc.BCError) as e:
        bc.plan_for_workload(w, to_device(w["fields"]),
                             stencil=bc.star_stencil(2, 1)).const_values(0)
    assert e.value.status == "BC_ERR_UNSUPPORTED"          # pruned


def test_tiny_cubed_sphere_full():
    """6 x 32^2, h = 2, p = 4, FP64 scalar, corners by CSR."""
    w = synth.tiny_cubed_sphere()
    plan, out = run(w)
    compare(w, out)
    assert plan.stats()["ghost_values"] == 6 * (36 * 36 - 32 * 32)


def test_swe_cubed_sphere_sampled():
    """6 x 384^2, h = 3, (h, u, v) x 32 levels FP32, p = 6: every ghost is
    computed on the GPU; levels 0, 13 and 31 are compared with the oracle."""
    w = synth.swe_cubed_sphere()
    _, out = run(w)
    compare(w, out, levels=[0, 13, 31])


def test_adjoint_config_forward_sampled():
    """6 x 768^2 forward, levels 5 and 30 compared."""
    w = synth.adjoint_cubed_sphere()
    _, out = run(w)
    compare(w, out, levels=[5, 30])


def test_export_csr_matches_oracle():
    """The plan's own rows of A (incl. the GPU-generated FP64 geometry)
    against the oracle's explicit A, entry by entry."""
    w = synth.cubed_sphere(12, 3, 6, 2, ("h", "u", "v"), "f64", seed=5)
    ts = to_device(w["fields"])
    plan = bc.plan_for_workload(w, ts)
    ex = plan.export_csr()
    op = build_operator(w, levels=[0])
    lay = op.layout
    # slot s = (block, comp) -> row/col ids of level 0
    slot_b, slot_c = [], []
    for b, blk in enumerate(w["blocks"]):
        for c in range(blk["ncomp"]):
            slot_b.append(b)
            slot_c.append(c)
    slot_b, slot_c = np.array(slot_b), np.array(slot_c)
    plane = lay.F.prod(axis=1)
    rows = lay.full_base[slot_b[ex["row_slot"]]] + \
        slot_c[ex["row_slot"]] * lay.L[slot_b[ex["row_slot"]]] * plane[slot_b[ex["row_slot"]]] + \
        ex["row_off"]
    assert np.array_equal(np.sort(rows), op.rows)
    # columns: full offset -> data cell -> column id
    cb = slot_b[ex["col_slot"]]
    F = lay.F[cb]
    h = lay.h[cb]
    o = ex["col_off"]
    i = o % F[:, 0] - h[:, 0]
    j = (o // F[:, 0]) % F[:, 1] - h[:, 1]
    k = o // (F[:, 0] * F[:, 1]) - h[:, 2]
    cols = lay.col(cb, slot_c[ex["col_slot"]], 0, np.stack([i, j, k], 1))
    import scipy.sparse as sp
    order = np.argsort(rows)
    A = sp.csr_matrix((ex["val"], cols, ex["row_ptr"]),
                      shape=(len(rows), lay.n_data))[order]
    A.sum_duplicates()
    D = (A - op.A).tocoo()
    assert A.nnz == op.A.nnz
    assert np.max(np.abs(D.data)) <= 1e-13 if D.nnz else True


def test_non_contiguous_layout():
    """Levels innermost: element (c, l, k, j, i) at ((c*F2 + k)*F1 + j)*F0*L
    + i*L + l; the plan takes the strides from the tensor views."""
    import torch
    w = synth.cubed_sphere(10, 2, 4, 5, ("h", "u", "v"), "f32", seed=9)
    views = []
    for a in w["fields"]:
        C, L, F2, F1, F0 = a.shape
        base = torch.from_numpy(np.ascontiguousarray(a.transpose(0, 2, 3, 4, 1))).cuda()
        views.append(base.permute(0, 4, 1, 2, 3))
    plan, _ = run(w, tensors=views)
    out = [v.cpu().numpy() for v in views]
    compare(w, out)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("form", FORMS)
def test_level_innermost_batching(dtype, form):
    """Levels contiguous in memory: every kind runs level-fastest."""
    w = synth.batching(nblocks=40, side_lo=3, side_hi=40, lev_lo=1, lev_hi=40,
                       h=2, seed=17, dtype=dtype)
    ts = to_device_innermost(w["fields"])
    _, _ = run(w, form=form, tensors=ts)
    compare(w, [t.cpu().numpy() for t in ts])


@pytest.mark.parametrize("N,L", [(9, 1), (16, 7), (12, 33)])
def test_level_innermost_cubed_sphere(N, L):
    w = synth.cubed_sphere(N, 3, 6, L, ("h", "u", "v"), "f32", seed=N)
    ts = to_device_innermost(w["fields"])
    run(w, tensors=ts)
    compare(w, [t.cpu().numpy() for t in ts])


def test_empty_plan():
    w = synth.alg1_example()
    w["bcs"] = []
    plan, out = run(w)
    assert np.array_equal(bits(flat(out)), bits(flat(w["fields"])))
    assert plan.stats()["nitems"] == 0


def test_graph_capture_replay():
    import torch
    w = synth.batching(nblocks=32, side_lo=4, side_hi=48, lev_lo=1, lev_hi=20,
                       h=2, seed=12, dtype="f32")
    ts = to_device(w["fields"])
    plan = bc.plan_for_workload(w, ts, {"ctas_per_sm": 2})
    table = bc.slot_table(ts)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.apply(table, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.apply(table, stream=s)
    for _ in range(100):
        g.replay()
    torch.cuda.synchronize()
    compare(w, [t.cpu().numpy() for t in ts])


def test_apply_host_roundtrip():
    import torch
    w = synth.batching(nblocks=16, side_lo=4, side_hi=32, lev_lo=1, lev_hi=9,
                       h=2, seed=13, dtype="f32")
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in w["fields"]]
    dev = [torch.empty_like(h, device="cuda") for h in host]
    plan = bc.plan_for_workload(w, dev)
    table = bc.slot_table(dev)
    plan.apply_host(bc.slot_pointers(host), bc.slot_pointers(dev), table)
    torch.cuda.synchronize()
    compare(w, [h.numpy() for h in host])


def test_copy_rows_preserve_nan_payload_and_signed_zero():
    """Copies move bit patterns: a NaN payload and -0.0 in the source data
    arrive unchanged in the ghosts that copy them."""
    w = synth.hpcg_block((6, 5, 4), "P", seed=1, dtype="f32")
    d = synth.data_view(w["fields"][0], w["blocks"][0])
    pay = np.array([0x7fc12345], np.uint32).view(np.float32)[0]
    d[0, 0, :, :, 5] = pay           # right x face: copied into the left ghosts
    d[0, 0, :, :, 0] = -0.0
    _, out = run(w)
    g = out[0][0, 0]
    assert np.all(bits(g[1:-1, 1:-1, 0]) == 0x7fc12345)
    assert np.all(bits(g[1:-1, 1:-1, -1]) == 0x80000000)


def test_autotune_keeps_results():
    import torch
    w = synth.batching(nblocks=64, side_lo=4, side_hi=64, lev_lo=1, lev_hi=40,
                       h=2, seed=14, dtype="f32")
    ts = to_device(w["fields"])
    plan = bc.plan_for_workload(w, ts)
    table = bc.slot_table(ts)
    plan.autotune(table)
    for t, a in zip(ts, w["fields"]):
        t.copy_(torch.from_numpy(a))
    plan.apply(table)
    torch.cuda.synchronize()
    compare(w, [t.cpu().numpy() for t in ts])


@pytest.mark.parametrize("layout", ["outermost", "innermost"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_runs_and_per_value_units_agree(layout, dtype):
    """Zero and map sub-matrices copy contiguous runs by default; with
    ``no_runs`` they use per-value units.  Both give the oracle's values bit
    for bit, forward and adjoint."""
    import torch
    w = synth.batching(nblocks=48, side_lo=3, side_hi=48, lev_lo=1, lev_hi=33,
                       h=2, seed=23, dtype=dtype)
    dev = to_device_innermost if layout == "innermost" else to_device
    outs, adjs = [], []
    cot = synth.cotangent_like(w, 24)
    for opts in ({}, {"no_runs": 1}):
        ts = dev(w["fields"])
        plan, _ = run(w, opts=opts, tensors=ts, repeat=2)
        outs.append(flat([t.cpu().numpy() for t in ts]))
        cs = dev(cot)
        plan.adjoint(bc.slot_table(cs))
        torch.cuda.synchronize()
        adjs.append(flat([c.cpu().numpy() for c in cs]))
    assert np.array_equal(bits(outs[0]), bits(outs[1]))
    assert np.array_equal(bits(adjs[0]), bits(adjs[1]))
    compare(w, [o for o in _unflat(outs[0], w["fields"])])


def _unflat(v, like):
    out, k = [], 0
    for a in like:
        out.append(v[k:k + a.size].reshape(a.shape))
        k += a.size
    return out


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["outermost", "innermost"])
def test_two_level_scaled_maps(dtype, layout):
    """Blocks of region steps 1 and 2: scale-2 injection maps and CSR
    prolongation rows, against the oracle (copies bit-exact)."""
    import torch
    w = synth.two_level(40, 26, 2, nlevels=5, ncomp=2, dtype=dtype, seed=14)
    ts = to_device_innermost(w["fields"]) if layout == "innermost" else to_device(w["fields"])
    run(w, tensors=ts)
    torch.cuda.synchronize()
    compare(w, [t.cpu().numpy() for t in ts])
