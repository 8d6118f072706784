"""CPU checks of the C ABI: the library builds and loads, exports every
function that include/bc.h declares, its ctypes structs match the header's
sizes, and invalid descriptions are rejected before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2605_14780_gb300 import bc, specs, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bc.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(bc.library_path()):
        from paper_2605_14780_gb300.build import build_library
        build_library()
    return bc.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(bc_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("bc_plan_create", "bc_apply", "bc_apply_adjoint",
              "bc_plan_destroy", "bc_status_string", "bc_last_error",
              "bc_plan_autotune", "bc_plan_export_csr"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert set(names) <= set(bc.SIGNATURES)
    for n in names:
        assert hasattr(lib, n), n


def test_struct_sizes_match_header():
    assert ctypes.sizeof(bc.BcBlock) == 64
    assert ctypes.sizeof(bc.BcPlanOpts) == 56
    # the sub-matrix struct: offsets of a few fields against the C layout
    assert bc.BcSubmatrix.comps.offset == 40
    assert bc.BcSubmatrix.row_ptr.offset > bc.BcSubmatrix.itp_rot.offset


def test_status_strings(lib):
    for code, name in bc.STATUS.items():
        assert lib.bc_status_string(code).decode() == name


def _expect(w, status, **kw):
    with pytest.raises(bc.BCError) as e:
        bc.plan_for_workload(w, **kw)
    assert e.value.status == status, str(e.value)


def test_rejects_overlap(lib):
    w = synth.alg1_example()
    w["bcs"].append({"kind": "zero", "block": 1, "lo": (5, 2, 0),
                     "hi": (6, 3, 1), "comps": [0]})
    _expect(w, "BC_ERR_OVERLAP")


def test_rejects_non_data_column(lib):
    w = synth.alg1_example()
    w["bcs"][0]["offset"] = (1, 9, 0)
    _expect(w, "BC_ERR_COLUMN_NOT_DATA")
    w = synth.alg1_example()
    w["bcs"][1]["col_ijk"] = w["bcs"][1]["col_ijk"].copy()
    w["bcs"][1]["col_ijk"][0] = (5, 0, 0)
    _expect(w, "BC_ERR_COLUMN_NOT_DATA")


def test_rejects_data_rows(lib):
    w = synth.alg1_example()
    w["bcs"].append({"kind": "zero", "block": 0, "lo": (0, 0, 0),
                     "hi": (1, 1, 1), "comps": [0]})
    _expect(w, "BC_ERR_OUT_OF_RANGE")


def test_rejects_too_deep_reflection(lib):
    blocks = [specs.contiguous_block(synth.block2d(3, 3, 2))]
    sub = {"kind": specs.BC_MAP, "block": 0, "lo": (-2, 0, 0), "hi": (0, 3, 1),
           "comps": [0], "src_block": 0, "perm": (0, 1, 2),
           "sign": (-1, 1, 1), "offset": (-1, 0, 0)}
    bc.Plan  # symbol exists
    # fine: depth 2 <= N = 3
    # too deep: N = 1 with h = 2
    blocks = [specs.contiguous_block(synth.block2d(1, 3, 2))]
    with pytest.raises(bc.BCError) as e:
        bc.Plan(blocks, [sub], "f32")
    assert e.value.status == "BC_ERR_HALO_TOO_WIDE"


def test_specs_reject_too_deep_faces():
    w = synth.hpcg_block((1, 4, 4), "P")
    w["blocks"][0]["h"] = (2, 2, 2)
    with pytest.raises(ValueError):
        specs.submatrices(w)


def test_rejects_bad_arguments(lib):
    w = synth.alg1_example()
    w["bcs"][2]["comps"] = [3]
    _expect(w, "BC_ERR_INVALID_ARG")
    w = synth.alg1_example()
    w["bcs"][0]["perm"] = (0, 0, 2)
    _expect(w, "BC_ERR_INVALID_ARG")
    w = synth.alg1_example()
    w["bcs"][1]["val"] = w["bcs"][1]["val"].copy()
    w["bcs"][1]["val"][2] = np.nan
    _expect(w, "BC_ERR_INVALID_ARG")


def test_strict_cover(lib):
    w = synth.alg1_example()
    _expect(w, "BC_ERR_UNCOVERED", opts={"strict_cover": 1})


def test_last_error_is_thread_local(lib):
    import threading
    w = synth.alg1_example()
    w["bcs"][0]["offset"] = (1, 9, 0)
    try:
        bc.plan_for_workload(w)
    except bc.BCError:
        pass
    msg = lib.bc_last_error().decode()
    assert "map image" in msg
    seen = []
    t = threading.Thread(target=lambda: seen.append(lib.bc_last_error().decode()))
    t.start()
    t.join()
    assert seen == [""]


def test_specs_halo_and_faces_cover_every_ghost():
    """The face decomposition is a partition of the ghost region."""
    w = synth.batching(nblocks=20, side_lo=3, side_hi=20, lev_lo=1, lev_hi=2,
                       h=2, seed=3)
    subs = specs.submatrices(w)
    cover = [np.zeros((b["n"][1] + 4, b["n"][0] + 4), int) for b in w["blocks"]]
    for s in subs:
        c = cover[s["block"]]
        c[s["lo"][1] + 2:s["hi"][1] + 2, s["lo"][0] + 2:s["hi"][0] + 2] += 1
    for b, c in zip(w["blocks"], cover):
        inner = c[2:2 + b["n"][1], 2:2 + b["n"][0]]
        assert np.all(inner == 0)
        c[2:2 + b["n"][1], 2:2 + b["n"][0]] = 1
        assert np.all(c == 1)


def _sync_workload():
    return synth.sync_grid(2, 2, 5, 1, nlevels=2, ncomp=1, dtype="f32", seed=3)


def test_rejects_sync_box_in_the_ghost_region(lib):
    w = _sync_workload()
    s = next(b for b in w["bcs"] if b["kind"] == "sync")
    n = w["blocks"][s["block"]]["n"]
    # move the box one cell past the data: its cells become ghosts
    hi = list(s["hi"])
    if s["lo"][0] == n[0] - 1:
        s["lo"], hi[0] = (n[0], s["lo"][1], 0), n[0] + 1
    else:
        s["lo"], hi[1] = (s["lo"][0], n[1], 0), n[1] + 1
    s["hi"] = tuple(hi)
    _expect(w, "BC_ERR_OUT_OF_RANGE")


def test_rejects_overlapping_sync_rows(lib):
    w = _sync_workload()
    s = next(b for b in w["bcs"] if b["kind"] == "sync")
    w["bcs"].append(dict(s))
    _expect(w, "BC_ERR_OVERLAP")


def test_rejects_sync_rows_with_a_constant(lib):
    w = _sync_workload()
    s = next(b for b in w["bcs"] if b["kind"] == "sync")
    s["rhs"] = np.full(len(s["row_ptr"]) - 1, 0.5)
    _expect(w, "BC_ERR_INVALID_ARG")


def test_rejects_sync_rows_reading_ghosts(lib):
    w = _sync_workload()
    s = next(b for b in w["bcs"] if b["kind"] == "sync")
    s["col_ijk"] = s["col_ijk"].copy()
    s["col_ijk"][0] = (-1, 0, 0)
    _expect(w, "BC_ERR_COLUMN_NOT_DATA")


def test_rejects_zero_map_scale(lib):
    w = synth.two_level(8, 6, 1, nlevels=1, ncomp=1, dtype="f32", seed=1)
    m = next(b for b in w["bcs"] if b["kind"] == "map")
    m["sign"] = (0, 2, 1)
    _expect(w, "BC_ERR_INVALID_ARG")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the compiled library the binding raises."""
    monkeypatch.setattr(bc, "_LIB", None)
    monkeypatch.setattr(bc, "library_path", lambda: str(tmp_path / "libbcgb300.so"))
    with pytest.raises(RuntimeError, match="not built"):
        bc.load_library()
    with pytest.raises(RuntimeError):
        bc.plan_for_workload(synth.alg1_example())


def test_tensor_layout_checks_on_the_host(lib):
    """The tensor API compares shape, dtype and strides with the layout the
    plan was built for before any device work (host-only plan, CPU
    tensors: the layout is right, so only the device is refused)."""
    import torch
    w = synth.batching(nblocks=6, side_lo=4, side_hi=12, lev_lo=2, lev_hi=6, h=2,
                       seed=5, dtype="f32")
    outer = [torch.from_numpy(a.copy()) for a in w["fields"]]
    inner = [torch.from_numpy(np.ascontiguousarray(a.transpose(0, 2, 3, 4, 1)))
             .permute(0, 4, 1, 2, 3) for a in w["fields"]]
    plan = bc.plan_for_workload(w, outer, {"host_only": 1})
    with pytest.raises(ValueError, match="stride"):
        plan.check_tensors(inner)
    with pytest.raises(ValueError, match="dtype"):
        plan.check_tensors([t.double() for t in outer])
    with pytest.raises(ValueError, match="shape"):
        plan.check_tensors([t[:, :1] for t in outer])
    with pytest.raises(ValueError, match="cuda|CUDA"):
        plan.check_tensors(outer)
    # a plan built on the level-innermost strides accepts those
    plan2 = bc.plan_for_workload(w, inner, {"host_only": 1})
    with pytest.raises(ValueError, match="CUDA"):
        plan2.check_tensors(inner)
    with pytest.raises(ValueError, match="stride"):
        plan2.check_tensors(outer)


@pytest.mark.parametrize("kind", ["circular", "symmetric"])
@pytest.mark.parametrize("axis,side", [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1)])
def test_fmap_submatrix_is_the_paper_map(lib, kind, axis, side):
    """bc_fmap_submatrix gives the face sub-matrix the Python face
    description builds (the paper's fmap, both sides; those rows are
    pinned against the oracle by the host-plan tests)."""
    w = synth.hpcg_block((5, 4, 6), "Z", seed=3)
    blk = w["blocks"][0]
    fm = bc.BC_FMAP_CIRCULAR if kind == "circular" else bc.BC_FMAP_SYMMETRIC
    sub = bc.fmap_submatrix([specs.contiguous_block(blk)], 0, axis, side, fm, [0])
    face = [s for s in specs.faces_submatrices(
        {"block": 0, "corners": "zero",
         "faces": [{"axis": a, "side": sd, "type": kind if (a, sd) == (axis, side) else "zero"}
                   for a in range(3) for sd in (0, 1)]}, w["blocks"])
        if s["kind"] == specs.BC_MAP]
    assert len(face) == 1
    for key in ("lo", "hi", "src_block", "perm", "sign", "offset"):
        assert tuple(np.atleast_1d(sub[key])) == tuple(np.atleast_1d(face[0][key])), key
    bad = dict(blk, h=(7, 1, 1))
    with pytest.raises(bc.BCError) as e:
        bc.fmap_submatrix([specs.contiguous_block(bad)], 0, 0, 0, fm, [0])
    assert e.value.status == "BC_ERR_HALO_TOO_WIDE"
