"""Pins of the oracle's rows that read other ghost values (the iterative form
HOPE(I) of Sec. II-B, folded into one matrix as HOPE(M) does).

* the oracle's single matrix equals a literal evaluation of the row sets,
  sweep by sweep, on the field (every ghost zero first);
* linear extrapolation faces reproduce a linear field exactly once the
  sweeps reach the ghost depth, and give the known partial values before;
* the contraction scheme after many sweeps satisfies every row equation
  (the fixed point of HOPE(I));
* one sweep is the same as dropping the ghost columns;
* a column on a ghost no sub-matrix covers is rejected.
"""
import numpy as np
import pytest

from oracle.operator import OracleError, apply, build_operator, rowsets
from oracle.regions import Layout
from paper_2605_14780_gb300 import synth


def _literal_sweeps(w, k):
    """k Jacobi sweeps straight from the row sets on the field values."""
    lay = Layout(w["blocks"])
    sets = rowsets(w)
    y = lay.flatten_full(w["fields"])
    covered = []
    for rs in sets:
        for lev in range(int(lay.L[rs["b"]])):
            rid = lay.row(np.full(len(rs["c"]), rs["b"]), rs["c"], lev, rs["ijk"])
            cid = lay.row(rs["e_b"], rs["e_c"], lev, rs["e_ijk"]) if len(rs["e_row"]) else None
            covered.append((rs, rid, cid))
    for _, rid, _ in covered:
        y[rid] = 0.0
    for _ in range(k):
        new = y.copy()
        for rs, rid, cid in covered:
            val = rs["rhs"].astype(np.float64).copy()
            if cid is not None:
                np.add.at(val, rs["e_row"], rs["e_w"] * y[cid])
            new[rid] = val
        y = new
    return y


@pytest.mark.parametrize("scheme", ["extrapolate", "smooth"])
@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_matrix_equals_literal_sweeps(scheme, k):
    w = synth.ghost_on_ghost(scheme=scheme, sweeps=k)
    op = build_operator(w)
    got = op.layout.flatten_full(apply(op, w["fields"]))
    ref = _literal_sweeps(w, k)
    assert np.allclose(got[op.rows], ref[op.rows], rtol=0, atol=1e-12)


def _linear_fields(w, alpha=0.75, beta=-1.25):
    lay = Layout(w["blocks"])
    out = []
    for blk, a in zip(w["blocks"], w["fields"]):
        n, h = blk["n"], blk["h"]
        jj, ii = np.meshgrid(np.arange(-h[1], n[1] + h[1]), np.arange(-h[0], n[0] + h[0]),
                             indexing="ij")
        full = np.empty_like(a)
        for c in range(a.shape[0]):
            for lev in range(a.shape[1]):
                full[c, lev, 0] = alpha * ii + beta * jj + 3.0 * c - lev
        out.append(full)
    return lay, out


def test_extrapolation_is_exact_after_h_sweeps():
    h = 3
    w = synth.ghost_on_ghost(h=h, scheme="extrapolate", sweeps=h)
    lay, exact = _linear_fields(w)
    w["fields"] = [e.copy() for e in exact]
    for a, blk in zip(w["fields"], w["blocks"]):
        n = blk["n"]
        a[:, :, :, :h, :] = np.nan
        a[:, :, :, n[1] + h:, :] = np.nan
        a[:, :, :, :, :h] = np.nan
        a[:, :, :, :, n[0] + h:] = np.nan
    op = build_operator(w)
    y = op.layout.flatten_full(apply(op, w["fields"]))
    ref = op.layout.flatten_full(exact)
    face = np.abs(op.A.sum(axis=1)).A1 > 0          # corner rows are zero rows
    assert np.allclose(y[op.rows][face], ref[op.rows][face], rtol=0, atol=1e-12)


def test_extrapolation_partial_values_after_one_sweep():
    """One sweep from zero ghosts: depth 0 = 2 x0 - x1, depth 1 = -x0,
    depth 2 = 0 (x0, x1 the first two data layers)."""
    w = synth.ghost_on_ghost(sizes=((6, 5),), h=3, nlevels=1, ncomp=1, scheme="extrapolate",
                             sweeps=1)
    y = apply(build_operator(w), w["fields"])[0][0, 0, 0]
    x = w["fields"][0][0, 0, 0]
    h = 3
    rows = slice(h, h + 5)
    x0, x1 = x[rows, h], x[rows, h + 1]           # low side of axis 0
    assert np.allclose(y[rows, h - 1], 2 * x0 - x1, rtol=0, atol=1e-15)
    assert np.allclose(y[rows, h - 2], -x0, rtol=0, atol=1e-15)
    assert np.all(y[rows, h - 3] == 0.0)


def test_contraction_reaches_the_fixed_point():
    """Many sweeps of the contraction: every row equation holds for the
    resulting ghosts (each row's sum of |G| entries is at most 0.5)."""
    w = synth.ghost_on_ghost(scheme="smooth", sweeps=120)
    op = build_operator(w)
    lay = op.layout
    y = lay.flatten_full(apply(op, w["fields"]))
    worst = 0.0
    for rs in rowsets(w):
        for lev in range(int(lay.L[rs["b"]])):
            rid = lay.row(np.full(len(rs["c"]), rs["b"]), rs["c"], lev, rs["ijk"])
            val = rs["rhs"].astype(np.float64).copy()
            if len(rs["e_row"]):
                cid = lay.row(rs["e_b"], rs["e_c"], lev, rs["e_ijk"])
                np.add.at(val, rs["e_row"], rs["e_w"] * y[cid])
            worst = max(worst, float(np.max(np.abs(y[rid] - val))))
    assert worst < 1e-12
    # and it is not the one-sweep answer
    w1 = dict(w, ghost_sweeps=1)
    y1 = lay.flatten_full(apply(build_operator(w1), w["fields"]))
    assert np.max(np.abs(y1[op.rows] - y[op.rows])) > 1e-3


@pytest.mark.parametrize("scheme", ["extrapolate", "smooth"])
def test_one_sweep_drops_the_ghost_columns(scheme):
    w = synth.ghost_on_ghost(scheme=scheme, sweeps=1)
    lay = Layout(w["blocks"])
    w0 = dict(w, ghost_sweeps=0, bcs=[])
    for bc in w["bcs"]:
        if bc["kind"] != "csr":
            w0["bcs"].append(bc)
            continue
        keep = lay.in_data(np.full(len(bc["val"]), bc["block"]), bc["col_ijk"])
        rp = bc["row_ptr"]
        cnt = np.add.reduceat(keep.astype(np.int64), rp[:-1]) if len(keep) else keep
        cnt = np.where(np.diff(rp) > 0, cnt, 0)
        d = dict(bc, row_ptr=np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64),
                 col_block=bc["col_block"][keep], col_comp=bc["col_comp"][keep],
                 col_ijk=bc["col_ijk"][keep], val=bc["val"][keep])
        w0["bcs"].append(d)
    a = build_operator(w)
    b = build_operator(w0)
    assert np.array_equal(a.rows, b.rows)
    assert abs(a.A - b.A).max() == 0.0 and np.array_equal(a.b, b.b)


def test_uncovered_ghost_column_is_rejected():
    """A row that reads the corner ghost (-1, -1) of block 0 is valid while
    the zero corner covers it and rejected once that corner is left out."""
    w = synth.ghost_on_ghost(scheme="extrapolate", sweeps=2)
    bc = w["bcs"][0]
    bc["col_ijk"] = bc["col_ijk"].copy()
    bc["col_ijk"][1] = (-1, -1, 0)
    build_operator(w)
    w["bcs"] = [d for d in w["bcs"]
                if not (d["kind"] == "zero" and d["block"] == 0 and tuple(d["hi"][:2]) == (0, 0))]
    with pytest.raises(OracleError):
        build_operator(w)
