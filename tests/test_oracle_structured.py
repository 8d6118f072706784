"""Pins of the oracle's structured rows (zero, maps, halo copies, CSR faces).

Each check compares the oracle with something other than itself: values the
paper prints (Alg. 1), closed forms, or numpy's own padding routines.
"""
import os

import numpy as np
import pytest

from oracle.operator import OracleError, apply, build_operator
from oracle.rows import fmap
from paper_2605_14780_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#", dtype=np.int64)


# ---------------------------------------------------------------------------
# fmap
# ---------------------------------------------------------------------------
def test_fmap_golden_N5():
    g = _load("fmap_N5.txt")
    assert np.array_equal(fmap(g[:, 0], 5, "symmetric"), g[:, 1])
    assert np.array_equal(fmap(g[:, 0], 5, "circular"), g[:, 2])


@pytest.mark.parametrize("N", range(1, 9))
def test_fmap_matches_numpy_pad(N):
    """Symmetric == numpy 'symmetric' padding, circular == 'wrap'."""
    for h in range(0, N + 1):
        idx = np.arange(-h, N + h)
        src = np.arange(N)
        assert np.array_equal(fmap(idx, N, "symmetric"),
                              np.pad(src, h, mode="symmetric"))
        assert np.array_equal(fmap(idx, N, "circular"),
                              np.pad(src, h, mode="wrap"))


def test_fmap_too_deep():
    with pytest.raises(OracleError):
        fmap(np.array([-4]), 3, "symmetric")
    with pytest.raises(OracleError):
        fmap(np.array([6]), 3, "circular")


# ---------------------------------------------------------------------------
# Alg. 1
# ---------------------------------------------------------------------------
def test_alg1_worked_example():
    w = synth.alg1_example()
    op = build_operator(w)
    lay = op.layout
    # 24 ghost cells of block 1 (7x7 - 5x5), none elsewhere
    assert len(op.rows) == 24
    assert np.all((op.rows >= lay.full_base[1]) & (op.rows < lay.full_base[2]))
    gold = _load("alg1_right_ghost.txt")
    for dst_b, d1, d2, src_b, s1, s2, val in gold:
        # paper index [block, idx1, idx2] -> (i = idx2, j = idx1)
        r = lay.row(np.array([dst_b]), 0, 0, np.array([[d2, d1, 0]]))[0]
        k = np.searchsorted(op.rows, r)
        assert op.rows[k] == r
        row = op.A.getrow(k)
        assert row.nnz == 1
        col = lay.col(np.array([src_b]), 0, 0, np.array([[s2, s1, 0]]))[0]
        assert row.indices[0] == col and row.data[0] == val
    # the zero rows: top and bottom ghost rows, corners included
    zero = 0
    for j in (-1, 5):
        for i in range(-1, 6):
            r = lay.row(np.array([1]), 0, 0, np.array([[i, j, 0]]))[0]
            k = np.searchsorted(op.rows, r)
            assert op.rows[k] == r and op.A.getrow(k).nnz == 0 and op.b[k] == 0
            zero += 1
    assert zero == 14
    # the left rows equal the user CSR entry for entry
    csr = [bc for bc in w["bcs"] if bc["kind"] == "csr"][0]
    for j in range(5):
        r = lay.row(np.array([1]), 0, 0, np.array([[-1, j, 0]]))[0]
        k = np.searchsorted(op.rows, r)
        row = op.A.getrow(k)
        lo, hi = csr["row_ptr"][j], csr["row_ptr"][j + 1]
        exp = {}
        for e in range(lo, hi):
            c = lay.col(np.array([0]), 0, 0, csr["col_ijk"][e][None, :])[0]
            exp[c] = exp.get(c, 0.0) + csr["val"][e]
        got = dict(zip(row.indices.tolist(), row.data.tolist()))
        assert got == exp


# ---------------------------------------------------------------------------
# 3-D faces with the product rule
# ---------------------------------------------------------------------------
def _pad_reference(data, variant):
    """Per-axis padding with numpy (x, then y, then z)."""
    modes = {"Z": ["constant"] * 3, "P": ["wrap", "constant", "constant"],
             "S": ["constant", "symmetric", "constant"]}[variant]
    out = data
    # data is (k, j, i): pad i (axis 2 of the array) first
    for axis_arr, mode in zip((2, 1, 0), modes):
        pw = [(0, 0)] * 3
        pw[axis_arr] = (1, 1)
        out = np.pad(out, pw, mode=mode) if mode != "constant" else \
            np.pad(out, pw, mode="constant", constant_values=0.0)
    return out


@pytest.mark.parametrize("variant", ["Z", "P", "S"])
@pytest.mark.parametrize("n", [(6, 6, 6), (7, 5, 4)])
def test_hpcg_faces_equal_numpy_padding(variant, n):
    w = synth.hpcg_block(n, variant, seed=7)
    op = build_operator(w)
    y = apply(op, w["fields"])[0][0, 0]
    data = synth.data_view(w["fields"][0], w["blocks"][0])[0, 0].astype(np.float64)
    ref = _pad_reference(data, variant)
    assert np.array_equal(y, ref)
    assert len(op.rows) == np.prod(np.array(n) + 2) - np.prod(n)


def _stencil27(full):
    out = 27.0 * full[1:-1, 1:-1, 1:-1]
    k, j, i = full.shape
    for dk in range(3):
        for dj in range(3):
            for di in range(3):
                out -= full[dk:k - 2 + dk, dj:j - 2 + dj, di:i - 2 + di]
    return out


@pytest.mark.parametrize("variant", ["Z", "P", "S"])
def test_hpcg_27point_closed_form(variant):
    gold = dict(_load("hpcg27_closed_form.txt").tolist())
    n = (9, 8, 7)
    w = synth.hpcg_block(n, variant, seed=3)
    d = synth.data_view(w["fields"][0], w["blocks"][0])
    d[...] = 1.0
    y = apply(build_operator(w), w["fields"])[0][0, 0]
    out = _stencil27(y)
    zero_axis = {"Z": (1, 1, 1), "P": (0, 1, 1), "S": (1, 0, 1)}[variant]
    kk, jj, ii = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]),
                             indexing="ij")
    touches = np.zeros(out.shape, np.int64)
    for ax, idx in zip((0, 1, 2), (ii, jj, kk)):
        at = (idx == 0) | (idx == n[ax] - 1)
        touches += at * zero_axis[ax]
    expect = np.vectorize(gold.get)(touches).astype(np.float64)
    assert np.array_equal(out, expect)


# ---------------------------------------------------------------------------
# 2-D faces of uneven blocks (halo, circular, symmetric, zero, CSR)
# ---------------------------------------------------------------------------
def _strip(arr2d, axis, side, h):
    """Data layers behind an edge as [depth r][along s] by slicing."""
    if axis == 0:
        lay = arr2d[:, :h] if side == 0 else arr2d[:, ::-1][:, :h]
        return lay.T
    lay = arr2d[:h, :] if side == 0 else arr2d[::-1, :][:h, :]
    return lay


def _ghost_strip(full2d, axis, side, h, n):
    """Ghost layers beyond an edge as [depth r][along s] by slicing."""
    nx, ny = n
    core_rows = full2d[h:h + ny, :]
    core_cols = full2d[:, h:h + nx]
    if axis == 0:
        g = core_rows[:, :h][:, ::-1] if side == 0 else core_rows[:, h + nx:]
        return g.T
    return core_cols[:h, :][::-1, :] if side == 0 else core_cols[h + ny:, :]


def test_batching_faces_by_slicing():
    w = synth.batching(nblocks=40, side_lo=4, side_hi=24, lev_lo=1, lev_hi=3,
                       h=2, seed=9, dtype="f64")
    y = apply(build_operator(w), w["fields"])
    seen = set()
    for bc in w["bcs"]:
        b = bc["block"]
        blk = w["blocks"][b]
        h = blk["h"][0]
        n = blk["n"][:2]
        for lev in range(blk["nlevels"]):
            full = y[b][0, lev, 0]
            data = synth.data_view(w["fields"][b], blk)[0, lev, 0].astype(np.float64)
            for f in bc["faces"]:
                got = _ghost_strip(full, f["axis"], f["side"], h, n)
                t = f["type"]
                seen.add(t)
                if t == "zero":
                    exp = np.zeros_like(got)
                elif t in ("circular", "symmetric"):
                    mode = "wrap" if t == "circular" else "symmetric"
                    pw = [(0, 0), (0, 0)]
                    pw[1 - f["axis"]] = (h, h)
                    padded = np.pad(data, pw, mode=mode)
                    full_ref = np.zeros((n[1] + 2 * h, n[0] + 2 * h))
                    if f["axis"] == 0:
                        full_ref[h:h + n[1], :] = padded
                    else:
                        full_ref[:, h:h + n[0]] = padded
                    exp = _ghost_strip(full_ref, f["axis"], f["side"], h, n)
                elif t == "halo":
                    sb = f["src_block"]
                    sblk = w["blocks"][sb]
                    sdata = synth.data_view(w["fields"][sb], sblk)[0, lev, 0]
                    exp = _strip(sdata.astype(np.float64), f["src_axis"],
                                 f["src_side"], h)
                    if f["flip"]:
                        exp = exp[:, ::-1]
                else:  # csr
                    lay = _strip(data, f["axis"], f["side"], 8)  # [layer][s]
                    exp = np.zeros_like(got)
                    for r in range(h):
                        for s in range(got.shape[1]):
                            k = f["nnz"][r, s]
                            acc = 0.0
                            for m in range(k):
                                acc += f["weights"][r, s, m] * lay[f["layers"][r, s, m], s]
                            exp[r, s] = acc
                    np.testing.assert_allclose(got, exp, rtol=1e-15, atol=1e-15)
                    continue
                assert np.array_equal(got, exp), (b, f)
            # corners are zero
            for cj in (slice(0, h), slice(h + n[1], None)):
                for ci in (slice(0, h), slice(h + n[0], None)):
                    assert np.all(full[cj, ci] == 0.0)
    assert seen == {"zero", "circular", "symmetric", "halo", "csr"}


# ---------------------------------------------------------------------------
# validation
# ---------------------------------------------------------------------------
def test_overlap_rejected():
    w = synth.alg1_example()
    w["bcs"].append({"kind": "zero", "block": 1, "lo": (5, 2, 0),
                     "hi": (6, 3, 1), "comps": [0]})
    with pytest.raises(OracleError):
        build_operator(w)


def test_non_data_column_rejected():
    w = synth.alg1_example()
    w["bcs"][0]["offset"] = (1, 9, 0)       # i' = j + 1 reaches i' = 5
    with pytest.raises(OracleError):
        build_operator(w)


def test_row_in_data_rejected():
    w = synth.alg1_example()
    w["bcs"].append({"kind": "zero", "block": 0, "lo": (0, 0, 0),
                     "hi": (1, 1, 1), "comps": [0]})
    with pytest.raises(OracleError):
        build_operator(w)


# ---------------------------------------------------------------------------
# planted mistakes must be caught by the pins above
# ---------------------------------------------------------------------------
def test_pin_catches_planted_fmap_error(monkeypatch):
    import oracle.rows as rows

    def bad(i, N, kind):
        out = np.asarray(i, np.int64).copy()
        out[out < 0] = -out[out < 0]        # off by one on the left side
        out[out >= N] = 2 * N - 1 - out[out >= N]
        return out
    monkeypatch.setattr(rows, "fmap", bad)
    w = synth.hpcg_block((6, 6, 6), "S", seed=7)
    y = apply(build_operator(w), w["fields"])[0][0, 0]
    data = synth.data_view(w["fields"][0], w["blocks"][0])[0, 0].astype(np.float64)
    assert not np.array_equal(y, _pad_reference(data, "S"))


def test_pure_function_boundary_closed_form():
    """Constant rows (A = 0, b = udf(i), Sec. III-B): every ghost value of the
    Dirichlet block equals the function at its cell, every data value is
    untouched."""
    t = 1.75
    w = synth.dirichlet_block(nx=9, ny=7, h=2, nlevels=2, ncomp=2, t=t)
    y = apply(build_operator(w), w["fields"])[0]
    C, L, _, F1, F0 = y.shape
    h = 2
    jj, ii = np.meshgrid(np.arange(F1) - h, np.arange(F0) - h, indexing="ij")
    ghost = (ii < 0) | (ii >= 9) | (jj < 0) | (jj >= 7)
    for c in range(C):
        for lev in range(L):
            want = 0.25 * ii - 0.5 * jj + 0.125 * t + c
            assert np.array_equal(y[c, lev, 0][ghost], want[ghost])
            assert np.array_equal(y[c, lev, 0][~ghost], w["fields"][0][c, lev, 0][~ghost])
