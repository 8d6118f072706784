"""The library's own plan construction on the CPU (host_only plans, no
device work): its explicit rows of A and b, read back with
bc_plan_export_csr, against the oracle's A and b for every workload type
except the GPU-generated cubed-sphere geometry -- maps, CSR, Sync rows,
scaled maps and pruned plans.  Pins the host half of the library (validation,
index maps, ELL packing, box cutting) without a GPU."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.operator import Operator, build_operator
from paper_2605_14780_gb300 import bc, synth
from pruning import live_mask

HOST = {"host_only": 1}


@pytest.fixture(autouse=True, scope="module")
def _library():
    import os
    if not os.path.exists(bc.library_path()):
        from paper_2605_14780_gb300.build import build_library
        build_library()


def _plan_matrix(w, plan):
    """(rows, A, b) of the plan in the oracle's numbering, level 0."""
    ex = plan.export_csr()
    op = build_operator(w, levels=[0])
    lay = op.layout
    slot_b, slot_c = [], []
    for b, blk in enumerate(w["blocks"]):
        for c in range(blk["ncomp"]):
            slot_b.append(b)
            slot_c.append(c)
    slot_b, slot_c = np.array(slot_b), np.array(slot_c)
    plane = lay.F.prod(axis=1)
    rb = slot_b[ex["row_slot"]]
    rows = lay.full_base[rb] + slot_c[ex["row_slot"]] * lay.L[rb] * plane[rb] + ex["row_off"]
    cb = slot_b[ex["col_slot"]]
    F, h, o = lay.F[cb], lay.h[cb], ex["col_off"]
    ijk = np.stack([o % F[:, 0] - h[:, 0], (o // F[:, 0]) % F[:, 1] - h[:, 1],
                    o // (F[:, 0] * F[:, 1]) - h[:, 2]], 1)
    cols = lay.col(cb, slot_c[ex["col_slot"]], 0, ijk)
    order = np.argsort(rows, kind="stable")
    A = sp.csr_matrix((ex["val"], cols, ex["row_ptr"]), shape=(len(rows), lay.n_data))[order]
    A.sum_duplicates()
    A.sort_indices()
    return rows[order], A, np.asarray(ex["rhs"])[order], op


def _same(rows, A, b, op):
    assert np.array_equal(rows, op.rows)
    assert A.nnz == op.A.nnz
    assert np.array_equal(A.indptr, op.A.indptr) and np.array_equal(A.indices, op.A.indices)
    assert np.allclose(A.data, op.A.data, rtol=0, atol=1e-15)
    assert np.allclose(b, op.b, rtol=0, atol=1e-15)


CASES = [
    ("alg1", lambda: synth.alg1_example(dtype="f64")),
    ("hpcg_Z", lambda: synth.hpcg_block((7, 5, 6), "Z", seed=1)),
    ("hpcg_P", lambda: synth.hpcg_block((7, 5, 6), "P", seed=1)),
    ("hpcg_S", lambda: synth.hpcg_block((6, 7, 5), "S", seed=2)),
    ("sync", lambda: synth.sync_grid(3, 2, 6, 2, 2, 2, "f64", seed=3)),
    ("two_level", lambda: synth.two_level(14, 10, 2, 2, 2, "f64", seed=4)),
] + [(f"batching{s}", (lambda s=s: synth.batching(
    nblocks=12, side_lo=2, side_hi=20, lev_lo=1, lev_hi=6, h=1 + s % 3, seed=s, dtype="f32")))
    for s in range(8)]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_host_plan_rows_equal_the_oracle(name, make):
    w = make()
    plan = bc.plan_for_workload(w, opts=HOST)
    _same(*_plan_matrix(w, plan))
    st = plan.stats()
    op_all = build_operator(w)
    assert st["ghost_values"] + st["sync_values"] == len(op_all.rows)


@pytest.mark.parametrize("stencil", [bc.star_stencil(2, 1), bc.box_stencil(2, 1),
                                     np.array([(1, 0, 0), (0, -2, 0)])])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_host_pruned_rows_are_the_live_rows(stencil, seed):
    w = synth.batching(nblocks=10, side_lo=2, side_hi=16, lev_lo=1, lev_hi=4, h=2,
                       seed=seed, dtype="f32")
    plan = bc.plan_for_workload(w, opts=HOST, stencil=stencil)
    rows, A, b, op = _plan_matrix(w, plan)
    keep = live_mask(w, stencil)[op.rows]
    _same(rows, A, b, Operator(op.layout, op.rows[keep], op.A[keep], op.b[keep]))


def test_host_plans_refuse_device_work():
    w = synth.alg1_example()
    plan = bc.plan_for_workload(w, opts=HOST)
    import ctypes
    st = plan._lib.bc_apply_form(plan._h, ctypes.c_void_p(1), 0, None)
    assert bc.STATUS.get(st) == "BC_ERR_UNSUPPORTED"
    with pytest.raises(bc.BCError) as e:
        bc.plan_for_workload(synth.tiny_cubed_sphere(), opts=HOST)
    assert e.value.status == "BC_ERR_UNSUPPORTED"


def test_algorithmic_bytes_closed_forms():
    """The roofline numerator: bc_plan_stats' forward bytes per ghost value
    are S for zero rows and 2S for copies (S = element size)."""
    for variant, per_value in (("Z", 1), ("P", None)):
        w = synth.hpcg_block((6, 5, 4), variant, seed=1, dtype="f64")
        st = bc.plan_for_workload(w, opts=HOST).stats()
        kinds = st["ghost_values_kind"]
        S = 8
        if per_value is not None:
            assert st["bytes_fwd"] == per_value * S * st["ghost_values"]
        else:
            # zero rows write S, map rows read and write S each
            assert st["bytes_fwd"] == S * kinds[0] + 2 * S * kinds[2]
    w = synth.sync_grid(2, 1, 5, 1, 3, 1, "f32", seed=2)
    st = bc.plan_for_workload(w, opts=HOST).stats()
    # the Sync rows (1 row per copy of the 5 shared nodes) at 3 levels
    assert st["sync_values"] == 2 * 5 * 3


@pytest.mark.parametrize("stencil", [bc.star_stencil(3, 1), bc.box_stencil(3, 1),
                                     np.array([(0, 0, 0), (1, 1, 0), (0, -1, 1)])])
@pytest.mark.parametrize("variant", ["Z", "P", "S"])
def test_host_pruned_3d(stencil, variant):
    w = synth.hpcg_block((6, 5, 4), variant, seed=3, dtype="f64")
    plan = bc.plan_for_workload(w, opts=HOST, stencil=stencil)
    rows, A, b, op = _plan_matrix(w, plan)
    keep = live_mask(w, stencil)[op.rows]
    _same(rows, A, b, Operator(op.layout, op.rows[keep], op.A[keep], op.b[keep]))


def _random_host_workload(seed):
    rng = np.random.default_rng(seed)
    kind = seed % 4
    dtype = ("f32", "f64")[int(rng.integers(2))]
    if kind == 0:
        h = int(rng.integers(1, 4))
        return synth.batching(nblocks=int(rng.integers(1, 16)), side_lo=h,
                              side_hi=int(rng.integers(h, 24)), lev_lo=1,
                              lev_hi=int(rng.integers(1, 9)), h=h, seed=seed, dtype=dtype)
    if kind == 1:
        return synth.sync_grid(int(rng.integers(1, 4)), int(rng.integers(1, 4)),
                               int(rng.integers(3, 8)), int(rng.integers(1, 3)),
                               int(rng.integers(1, 4)), int(rng.integers(1, 3)), dtype, seed=seed)
    if kind == 2:
        return synth.two_level(2 * int(rng.integers(2, 9)), 2 * int(rng.integers(2, 8)),
                               int(rng.integers(1, 3)), int(rng.integers(1, 4)),
                               int(rng.integers(1, 3)), dtype, seed=seed)
    n = tuple(int(x) for x in rng.integers(2, 7, size=3))
    return synth.hpcg_block(n, "ZPS"[int(rng.integers(3))], seed=seed, dtype=dtype)


@pytest.mark.parametrize("seed", range(40))
def test_host_plan_random_sweep(seed):
    """40 seeded random workloads, plain and pruned for a random stencil."""
    w = _random_host_workload(seed)
    rng = np.random.default_rng(100 + seed)
    plan = bc.plan_for_workload(w, opts=HOST)
    _same(*_plan_matrix(w, plan))
    n, bad, msg = plan.check_work()
    assert bad == 0, msg
    ndim = 3 if w["blocks"][0]["n"][2] > 1 else 2
    offs = rng.integers(-2, 3, size=(int(rng.integers(1, 6)), 3))
    if ndim == 2:
        offs[:, 2] = 0
    plan = bc.plan_for_workload(w, opts=HOST, stencil=offs.astype(np.int32))
    rows, A, b, op = _plan_matrix(w, plan)
    keep = live_mask(w, offs)[op.rows]
    # Sync rows (data cells) are kept by a pruned plan whatever the stencil
    datarow = np.zeros(live_mask(w, offs).size, bool)
    datarow[op.layout.data_rows()] = True
    keep |= datarow[op.rows]
    _same(rows, A, b, Operator(op.layout, op.rows[keep], op.A[keep], op.b[keep]))


# -- reconstruction-and-quadrature cubed-sphere rows (built on the host) --------
def _close(rows, A, b, op, atol=1e-13):
    """Same rows and sparsity; weights within FP64 rounding of the oracle
    (the rows are sums of products computed in another order)."""
    assert np.array_equal(rows, op.rows)
    assert np.array_equal(A.indptr, op.A.indptr) and np.array_equal(A.indices, op.A.indices)
    assert np.allclose(A.data, op.A.data, rtol=0, atol=atol)
    assert np.allclose(b, op.b, rtol=0, atol=1e-15)


QUAD_CASES = [(8, 2, 4, 2, ("h", "u", "v"), "f64"), (9, 3, 3, 1, ("scalar",), "f32"),
              (10, 1, 6, 3, ("h", "u", "v"), "f32"), (12, 3, 8, 4, ("scalar",), "f64"),
              (6, 2, 2, 8, ("h", "u", "v"), "f64"), (7, 3, 5, 2, ("h", "u", "v"), "f64"),
              (5, 1, 2, 5, ("scalar",), "f64"), (6, 2, 3, 6, ("h", "u", "v"), "f32"),
              (8, 1, 7, 7, ("scalar",), "f64")]


@pytest.mark.parametrize("N,h,p,nq,fields,dtype", QUAD_CASES)
def test_host_quadrature_rows_equal_the_oracle(N, h, p, nq, fields, dtype):
    w = synth.cubed_sphere(N, h, p, 2, fields, dtype, seed=5, quad=nq)
    plan = bc.plan_for_workload(w, opts=HOST)
    _close(*_plan_matrix(w, plan))
    st = plan.stats()
    # every edge ghost is a CSR row of p^2 (scalar) or 2 p^2 (vector) entries
    assert st["ghost_values_kind"][3] == 0
    assert st["ghost_values"] == len(build_operator(w).rows)


@pytest.mark.parametrize("stencil", [bc.star_stencil(2, 1), bc.box_stencil(2, 2)])
def test_host_quadrature_pruned(stencil):
    w = synth.cubed_sphere(9, 3, 4, 1, ("h", "u", "v"), "f64", seed=6, quad=2)
    plan = bc.plan_for_workload(w, opts=HOST, stencil=stencil)
    rows, A, b, op = _plan_matrix(w, plan)
    keep = live_mask(w, stencil)[op.rows]
    _close(rows, A, b, Operator(op.layout, op.rows[keep], op.A[keep], op.b[keep]))


def _quad_subs(**change):
    from paper_2605_14780_gb300 import specs
    w = synth.cubed_sphere(6, 2, 4, 1, ("h", "u", "v"), "f64", seed=7, quad=2)
    subs = specs.submatrices(w)
    subs[0].update(change)
    return w, subs


@pytest.mark.parametrize("change,status", [
    ({"nquad": 0}, "BC_ERR_UNSUPPORTED"), ({"nquad": 9}, "BC_ERR_UNSUPPORTED"),
    ({"p": 1}, "BC_ERR_UNSUPPORTED"), ({"p": 9}, "BC_ERR_UNSUPPORTED"),
    ({"p": 7}, "BC_ERR_INVALID_ARG"),                       # wider than N = 6
    ({"rot_comp": (1, 1)}, "BC_ERR_INVALID_ARG"), ({"rot_comp": (1, -1)}, "BC_ERR_INVALID_ARG"),
    ({"comps": [0, 1, 2, 3]}, "BC_ERR_INVALID_ARG"),
    ({"cs_panels": (0, 1, 2, 3, 4, 6)}, "BC_ERR_INVALID_ARG"),
    ({"lo": (-2, -1, 0)}, "BC_ERR_GEOMETRY"),               # a corner ghost in the box
    ({"lo": (-2, 0, 0), "hi": (1, 6, 1)}, "BC_ERR_GEOMETRY"),  # a data cell in the box
    ({"lo": (-3, 0, 0)}, "BC_ERR_OUT_OF_RANGE"),            # deeper than h = 2
    ({"hi": (0, 1 << 20, 1)}, "BC_ERR_OUT_OF_RANGE"),
])
def test_host_quadrature_rejects(change, status):
    w, subs = _quad_subs(**change)
    from paper_2605_14780_gb300 import specs
    blocks = [specs.contiguous_block(b) for b in w["blocks"]]
    with pytest.raises(bc.BCError) as e:
        bc.Plan(blocks, subs, w["dtype"], opts=HOST)
    assert e.value.status == status, e.value


@pytest.mark.parametrize("seed", range(12))
def test_host_quadrature_random(seed):
    """Random order, Gauss points, halo and fields; plain and pruned to a
    random stencil."""
    rng = np.random.default_rng(900 + seed)
    N = int(rng.integers(4, 15))
    h = int(rng.integers(1, min(3, N // 2) + 1))
    p = int(rng.integers(2, min(8, N) + 1))
    fields = (("scalar",), ("h", "u", "v"))[int(rng.integers(2))]
    w = synth.cubed_sphere(N, h, p, int(rng.integers(1, 4)), fields,
                           ("f32", "f64")[int(rng.integers(2))], seed=seed,
                           quad=int(rng.integers(1, 9)))
    _close(*_plan_matrix(w, bc.plan_for_workload(w, opts=HOST)))
    offs = rng.integers(-2, 3, size=(int(rng.integers(1, 6)), 3))
    offs[:, 2] = 0
    rows, A, b, op = _plan_matrix(w, bc.plan_for_workload(w, opts=HOST,
                                                          stencil=offs.astype(np.int32)))
    keep = live_mask(w, offs)[op.rows]
    _close(rows, A, b, Operator(op.layout, op.rows[keep], op.A[keep], op.b[keep]))


def test_host_plan_has_no_constant_tables():
    w = synth.dirichlet_block(t=1.5)
    plan = bc.plan_for_workload(w, opts=HOST)
    _same(*_plan_matrix(w, plan))
    with pytest.raises(bc.BCError) as e:
        plan.const_values(0)
    assert e.value.status == "BC_ERR_UNSUPPORTED"


# -- rows that read ghost values, folded by Jacobi sweeps ----------------------
@pytest.mark.parametrize("scheme", ["extrapolate", "smooth"])
@pytest.mark.parametrize("k", [1, 2, 3, 7])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_host_ghost_sweeps_equal_the_oracle(scheme, k, dtype):
    w = synth.ghost_on_ghost(scheme=scheme, sweeps=k, dtype=dtype)
    _close(*_plan_matrix(w, bc.plan_for_workload(w, opts=HOST)), atol=1e-14)


@pytest.mark.parametrize("stencil", [bc.star_stencil(2, 1), bc.box_stencil(2, 2)])
def test_host_ghost_sweeps_pruned(stencil):
    """Folding sees every row; pruning then keeps the live ones."""
    w = synth.ghost_on_ghost(scheme="smooth", sweeps=4)
    rows, A, b, op = _plan_matrix(w, bc.plan_for_workload(w, opts=HOST, stencil=stencil))
    keep = live_mask(w, stencil)[op.rows]
    _close(rows, A, b, Operator(op.layout, op.rows[keep], op.A[keep], op.b[keep]), atol=1e-14)


def test_host_ghost_sweeps_rejects():
    w = synth.ghost_on_ghost(scheme="extrapolate", sweeps=2)
    for k, status in ((-1, "BC_ERR_INVALID_ARG"), (65, "BC_ERR_INVALID_ARG"),
                      (0, "BC_ERR_COLUMN_NOT_DATA")):
        with pytest.raises(bc.BCError) as e:
            bc.plan_for_workload(dict(w, ghost_sweeps=None), opts=dict(HOST, ghost_sweeps=k))
        assert e.value.status == status, (k, e.value)
    # a column on a ghost that no sub-matrix covers
    w2 = synth.ghost_on_ghost(scheme="extrapolate", sweeps=2)
    w2["bcs"][0]["col_ijk"] = w2["bcs"][0]["col_ijk"].copy()
    w2["bcs"][0]["col_ijk"][1] = (-1, -1, 0)
    w2["bcs"] = [d for d in w2["bcs"] if not (d["kind"] == "zero" and d["block"] == 0
                                               and tuple(d["hi"][:2]) == (0, 0))]
    with pytest.raises(bc.BCError) as e:
        bc.plan_for_workload(w2, opts=HOST)
    assert e.value.status == "BC_ERR_COLUMN_NOT_DATA"
    # GPU-generated cubed-sphere rows cannot be folded on the host
    t = synth.tiny_cubed_sphere()
    with pytest.raises(bc.BCError) as e:
        bc.plan_for_workload(dict(t, ghost_sweeps=2), opts=HOST)
    assert e.value.status == "BC_ERR_UNSUPPORTED" and "fold" in str(e.value)


def _close_values(rows, A, b, op, atol=1e-13):
    """Same rows, entries equal within FP64 rounding (an entry that cancels
    to zero on one side may be stored or dropped on the other)."""
    assert np.array_equal(rows, op.rows)
    assert abs(A - op.A).max() <= atol if A.nnz + op.A.nnz else True
    assert np.allclose(b, op.b, rtol=0, atol=1e-14)


@pytest.mark.parametrize("N,h,p,nq,k,fields,dtype", [
    (12, 3, 4, 2, 10, ("h", "u", "v"), "f64"), (9, 2, 4, 1, 3, ("scalar",), "f32"),
    (10, 3, 6, 3, 2, ("h", "u", "v"), "f64"), (8, 1, 2, 2, 5, ("scalar",), "f64")])
def test_host_centred_quadrature_folded(N, h, p, nq, k, fields, dtype):
    """Centred patches read the neighbour's ghost cells (HOPE(I)); folded
    by k sweeps, the library's rows equal the oracle's."""
    w = synth.cubed_sphere(N, h, p, 2, fields, dtype, seed=5, quad=nq, centred=True, sweeps=k)
    _close_values(*_plan_matrix(w, bc.plan_for_workload(w, opts=HOST)))


def test_host_centred_quadrature_needs_sweeps():
    w = synth.cubed_sphere(8, 2, 4, 1, ("scalar",), "f64", seed=5, quad=2, centred=True)
    with pytest.raises(bc.BCError) as e:
        bc.plan_for_workload(dict(w, ghost_sweeps=None), opts=HOST)
    assert e.value.status == "BC_ERR_COLUMN_NOT_DATA"
    w = synth.cubed_sphere(8, 1, 6, 1, ("scalar",), "f64", seed=5, quad=2, centred=True)
    with pytest.raises(bc.BCError) as e:                     # h < p/2: patch leaves the region
        bc.plan_for_workload(w, opts=HOST)
    assert e.value.status == "BC_ERR_GEOMETRY"


@pytest.mark.parametrize("n,variant", [((1, 1, 1), "P"), ((1, 1, 1), "S"), ((1, 2, 1), "Z"),
                                       ((2, 1, 3), "P")])
def test_host_degenerate_block_sizes(n, variant):
    """One-cell extents: circular and symmetric maps of a single data layer
    (h = N = 1), and blocks of one cell along some axes."""
    w = synth.hpcg_block(n, variant, seed=3)
    _same(*_plan_matrix(w, bc.plan_for_workload(w, opts=HOST)))


def test_host_tiny_uneven_blocks():
    w = synth.batching(nblocks=6, side_lo=1, side_hi=3, lev_lo=1, lev_hi=3, h=1, seed=5,
                       dtype="f64")
    assert min(min(b["n"][:2]) for b in w["blocks"]) == 1
    _same(*_plan_matrix(w, bc.plan_for_workload(w, opts=HOST)))


def test_host_largest_component_span():
    """Element offsets are 32-bit: the largest element offset of a component
    must stay below 2^31 - 1 (here set through a padded axis-2 stride: the
    last cell sits at 15 + 3 s2)."""
    from paper_2605_14780_gb300 import specs
    s_max = (2 ** 31 - 2 - 15) // 3
    for s2, ok in ((s_max, True), (s_max + 1, False)):
        blk = {"n": (2, 2, 2), "h": (1, 1, 1), "nlevels": 1, "ncomp": 1,
               "stride": (1, 4, s2), "level_stride": 1}
        subs = [specs._sub(specs.BC_ZERO, 0, (-1, 0, 0), (0, 2, 2), [0])]
        if ok:
            plan = bc.Plan([blk], subs, "f64", opts=HOST)
            assert plan.stats()["ghost_values"] == 4
        else:
            with pytest.raises(bc.BCError) as e:
                bc.Plan([blk], subs, "f64", opts=HOST)
            assert e.value.status == "BC_ERR_UNSUPPORTED"


# -- host replay of the work lists ---------------------------------------------
def _innermost_blocks(w):
    """Block descriptors with the levels of every cell contiguous."""
    out = []
    for b in w["blocks"]:
        n, h, L = b["n"], b["h"], b["nlevels"]
        F = [n[d] + 2 * h[d] for d in range(3)]
        out.append({"n": tuple(n), "h": tuple(h), "nlevels": L, "ncomp": b["ncomp"],
                    "stride": (L, L * F[0], L * F[0] * F[1]), "level_stride": 1})
    return out


WORK_CASES = [
    ("alg1", lambda: synth.alg1_example()),
    ("hpcg_P", lambda: synth.hpcg_block((7, 5, 6), "P", seed=1)),
    ("batching", lambda: synth.batching(nblocks=16, side_lo=2, side_hi=40, lev_lo=1, lev_hi=20,
                                        h=2, seed=3, dtype="f32")),
    ("sync", lambda: synth.sync_grid(3, 2, 6, 2, 3, 2, "f64", seed=3)),
    ("two_level", lambda: synth.two_level(14, 10, 2, 3, 2, "f64", seed=4)),
    ("quadrature", lambda: synth.cubed_sphere(8, 2, 4, 5, ("h", "u", "v"), "f32", seed=5, quad=2)),
    ("ghost", lambda: synth.ghost_on_ghost(scheme="smooth", sweeps=4, nlevels=3)),
    ("dirichlet", lambda: synth.dirichlet_block(nlevels=9)),
    ("user_interp", lambda: synth.staggered_interp(nlevels=5)),
]
WORK_OPTS = [{}, {"no_runs": 1}, {"units_per_lane": 1}, {"units_per_lane": 8, "unit_order": 1},
             {"unit_order": 2}, {"threads": 512, "units_per_lane": 2}]


@pytest.mark.parametrize("name,make", WORK_CASES, ids=[c[0] for c in WORK_CASES])
@pytest.mark.parametrize("opts", WORK_OPTS, ids=lambda o: "-".join(f"{k}{v}" for k, v in o.items())
                         or "default")
@pytest.mark.parametrize("layout", ["outermost", "innermost"])
def test_work_lists_replay_against_rows(name, make, opts, layout):
    """Every forward item (per-kind and batched lists) and adjoint item,
    replayed on the host with the kernels' unit decompositions, writes each
    covered value once with its row's source or value, and each data value
    gathers exactly its A^T terms."""
    from paper_2605_14780_gb300 import specs
    w = make()
    o = dict(HOST, **opts)
    if w.get("ghost_sweeps"):
        o["ghost_sweeps"] = w["ghost_sweeps"]
    blocks = (_innermost_blocks(w) if layout == "innermost"
              else [specs.contiguous_block(b) for b in w["blocks"]])
    plan = bc.Plan(blocks, specs.submatrices(w), w["dtype"], o)
    n, bad, msg = plan.check_work()
    assert n > 0 and bad == 0, msg


@pytest.mark.parametrize("opts", [{}, {"level_chunk": 4}, {"batch_mode": bc.BC_BATCH_SINGLE},
                                  {"threads": 512}])
def test_staged_tiles_replay_against_rows(opts):
    """Levels outermost, reconstruction-and-quadrature rows on a 6 x 24^2
    sphere: the plan stages CSR tiles (16-row tiles where 32 rows' boxes are
    too large) and transpose tiles; every staged entry's box word, replayed
    on the host, names its row's column, with the per-lane plan as the
    control (fewer items)."""
    from paper_2605_14780_gb300 import specs
    w = synth.cubed_sphere(24, 3, 4, 9, ("h", "u", "v"), "f32", seed=41, quad=2)
    blocks = [specs.contiguous_block(b) for b in w["blocks"]]
    stats = []
    for unstaged in (0, 1):
        plan = bc.Plan(blocks, specs.submatrices(w), w["dtype"],
                       dict(HOST, unstaged_rows=unstaged, **opts))
        n, bad, msg = plan.check_work()
        assert n > 0 and bad == 0, msg
        st = plan.stats()
        stats.append((st["nitems"], st["nitems_adjoint"]))
    assert stats[0][0] != stats[1][0] and stats[0][1] != stats[1][1]


@pytest.mark.parametrize("stencil", [bc.star_stencil(2, 1), bc.box_stencil(2, 2)])
def test_work_lists_of_pruned_plans(stencil):
    w = synth.batching(nblocks=12, side_lo=2, side_hi=30, lev_lo=1, lev_hi=9, h=2, seed=6,
                       dtype="f32")
    n, bad, msg = bc.plan_for_workload(w, opts=HOST, stencil=stencil).check_work()
    assert n > 0 and bad == 0, msg


@pytest.mark.parametrize("plant", ["drop", "dup", "adjdrop"])
def test_work_replay_catches_planted_mistakes(monkeypatch, plant):
    """The replay alters its own copies of the lists (never the plan): a
    dropped item, a duplicated item and a dropped adjoint item are found."""
    w = synth.batching(nblocks=8, side_lo=2, side_hi=20, lev_lo=1, lev_hi=6, h=2, seed=3,
                       dtype="f32")
    plan = bc.plan_for_workload(w, opts=HOST)
    assert plan.check_work()[1] == 0
    monkeypatch.setenv("BC_CHECK_PLANT", plant)
    n, bad, msg = plan.check_work()
    assert bad > 0 and msg


@pytest.mark.parametrize("p", [2, 4, 6])
@pytest.mark.parametrize("rotate", [True, False])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_host_user_interpolation_tables(p, rotate, dtype):
    """Interpolation rows given as user tables (geometry BC_GEOM_USER)."""
    w = synth.staggered_interp(p=p, rotate=rotate, dtype=dtype)
    _same(*_plan_matrix(w, bc.plan_for_workload(w, opts=HOST)))


def test_host_user_interpolation_along_axis_0():
    w = synth.swap_xy(synth.staggered_interp(nx=11, ny=9, p=4))
    plan = bc.plan_for_workload(w, opts=HOST)
    _same(*_plan_matrix(w, plan))
    assert plan.check_work()[1] == 0


def test_host_user_interpolation_rejects():
    from paper_2605_14780_gb300 import specs
    w = synth.staggered_interp()
    blocks = [specs.contiguous_block(b) for b in w["blocks"]]
    for change, status in (
            ({"itp_w": None}, "BC_ERR_INVALID_ARG"),                 # tables missing
            ({"itp_axis": np.full(24, 3, np.int32)}, "BC_ERR_INVALID_ARG"),
            ({"p": 9}, "BC_ERR_UNSUPPORTED")):
        subs = specs.submatrices(w)
        subs[0] = dict(subs[0], **change)
        with pytest.raises(bc.BCError) as e:
            bc.Plan(blocks, subs, w["dtype"], opts=HOST)
        assert e.value.status == status, (change, e.value)
    # a stencil that leaves the source data
    subs = specs.submatrices(w)
    st = np.asarray(subs[0]["itp_start"]).reshape(-1, 3).copy()
    st[0, 1] = 12 - 2                                            # rows 10..13 of 12
    subs[0] = dict(subs[0], itp_start=st.reshape(-1))
    with pytest.raises(bc.BCError) as e:
        bc.Plan(blocks, subs, w["dtype"], opts=HOST)
    assert e.value.status == "BC_ERR_COLUMN_NOT_DATA"
