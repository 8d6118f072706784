"""Pins of the oracle's assembly, apply and adjoint.

The adjoint is checked against central finite differences of the *forward*
apply (a separate code path from the transpose), the dot-product identity is
evaluated with compensated sums, and explicit CSR rows must equal the user's
matrix entry for entry.
"""

import numpy as np
import pytest

from oracle.operator import apply, apply_adjoint, build_operator, row_scale
from paper_2605_14780_gb300 import synth


def _workloads():
    yield synth.alg1_example()
    yield synth.hpcg_block((5, 4, 6), "P", seed=1)
    yield synth.hpcg_block((5, 4, 6), "S", seed=1)
    yield synth.batching(nblocks=12, side_lo=4, side_hi=12, lev_lo=1,
                         lev_hi=3, h=2, seed=5, dtype="f64")
    yield synth.cubed_sphere(6, 2, 4, 2, ("h", "u", "v"), "f64", seed=3)


def _flat(arrs):
    return np.concatenate([np.asarray(a, np.float64).ravel() for a in arrs])


def _dot_compensated(a, b):
    """Neumaier-compensated sum of a*b and the sum of |a*b|."""
    s, c, mag = 0.0, 0.0, 0.0
    for v in (np.asarray(a) * np.asarray(b)).tolist():
        t = s + v
        if abs(s) >= abs(v):
            c += (s - t) + v
        else:
            c += (v - t) + s
        s = t
        mag += abs(v)
    return s + c, mag


@pytest.mark.parametrize("wi", range(5))
def test_adjoint_against_forward_fd(wi):
    w = list(_workloads())[wi]
    op = build_operator(w)
    rng = np.random.default_rng(100 + wi)
    cot = synth.cotangent_like(w, 200 + wi)
    xbar = _flat(apply_adjoint(op, cot))
    for _ in range(8):
        dirs = [np.where(np.isnan(a), 0.0, rng.uniform(-1, 1, a.shape))
                for a in w["fields"]]
        # the direction only moves data cells; ghosts are outputs
        for blk, dd in zip(w["blocks"], dirs):
            n, h = blk["n"], blk["h"]
            mask = np.ones(dd.shape, bool)
            mask[:, :, h[2]:h[2] + n[2], h[1]:h[1] + n[1], h[0]:h[0] + n[0]] = False
            dd[mask] = 0.0
        eps = 0.5
        xp = [np.where(np.isnan(a), 0.0, a) + eps * d for a, d in zip(w["fields"], dirs)]
        xm = [np.where(np.isnan(a), 0.0, a) - eps * d for a, d in zip(w["fields"], dirs)]
        jd = (_flat(apply(op, xp)) - _flat(apply(op, xm))) / (2 * eps)
        lhs, m1 = _dot_compensated(_flat(cot), jd)
        rhs, m2 = _dot_compensated(xbar, _flat(dirs))
        assert abs(lhs - rhs) <= 1e-13 * max(m1, m2)


@pytest.mark.parametrize("wi", range(5))
def test_dot_product_identity(wi):
    """<A x, y> == <x, A^T y> on the ghost rows, compensated sums."""
    w = list(_workloads())[wi]
    op = build_operator(w)
    rng = np.random.default_rng(wi)
    x = rng.uniform(-1, 1, op.layout.n_data)
    y = rng.uniform(-1, 1, len(op.rows))
    ax = np.array([op.A.getrow(i).dot(x)[0] for i in range(op.A.shape[0])]) \
        if op.A.shape[0] < 2000 else op.A @ x
    lhs, m1 = _dot_compensated(ax, y)
    aty = op.A.T @ y
    rhs, m2 = _dot_compensated(x, aty)
    assert abs(lhs - rhs) <= 1e-13 * max(m1, m2)


def test_adjoint_zeroes_covered_ghosts_only():
    w = synth.alg1_example()
    op = build_operator(w)
    cot = synth.cotangent_like(w, 3)
    out = apply_adjoint(op, cot)
    # blocks 0 and 2 have no ghost rows: their ghosts pass through
    for b in (0, 2):
        blk = w["blocks"][b]
        n, h = blk["n"], blk["h"]
        g = np.ones(cot[b].shape, bool)
        g[:, :, :, h[1]:h[1] + n[1], h[0]:h[0] + n[0]] = False
        assert np.array_equal(out[b][g], cot[b][g].astype(np.float64))
    # block 1's ghosts are all covered: zero
    blk = w["blocks"][1]
    g = np.ones(cot[1].shape, bool)
    g[:, :, :, 1:6, 1:6] = False
    assert np.all(out[1][g] == 0.0)


def test_csr_rows_equal_user_matrix():
    w = synth.cubed_sphere(6, 2, 4, 1, ("h", "u", "v"), "f64", seed=3)
    op = build_operator(w)
    lay = op.layout
    for bc in w["bcs"]:
        if bc["kind"] != "csr":
            continue
        lo, hi = bc["lo"], bc["hi"]
        vol = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
        r = 0
        for c in bc["comps"]:
            for k in range(lo[2], hi[2]):
                for j in range(lo[1], hi[1]):
                    for i in range(lo[0], hi[0]):
                        rid = lay.row(np.array([bc["block"]]), c, 0,
                                      np.array([[i, j, k]]))[0]
                        pos = np.searchsorted(op.rows, rid)
                        row = op.A.getrow(pos)
                        exp = {}
                        for e in range(bc["row_ptr"][r], bc["row_ptr"][r + 1]):
                            col = lay.col(np.array([bc["col_block"][e]]),
                                          bc["col_comp"][e], 0,
                                          bc["col_ijk"][e][None, :])[0]
                            exp[col] = exp.get(col, 0.0) + bc["val"][e]
                        assert dict(zip(row.indices.tolist(),
                                        row.data.tolist())) == exp
                        r += 1
        assert r == len(bc["comps"]) * vol


def test_levels_restriction_matches_full():
    w = synth.batching(nblocks=8, side_lo=4, side_hi=10, lev_lo=2, lev_hi=5,
                       h=2, seed=1, dtype="f64")
    full = build_operator(w)
    part = build_operator(w, levels=[1])
    gfull = full.A @ full.layout.data_vector(w["fields"]) + full.b
    gpart = part.A @ part.layout.data_vector(w["fields"]) + part.b
    idx = np.searchsorted(full.rows, part.rows)
    assert np.array_equal(full.rows[idx], part.rows)
    assert np.array_equal(gfull[idx], gpart)


def test_row_scale_bounds_values():
    w = synth.cubed_sphere(6, 2, 4, 2, ("h", "u", "v"), "f64", seed=3)
    op = build_operator(w)
    g = op.A @ op.layout.data_vector(w["fields"]) + op.b
    s = row_scale(op, w["fields"])
    assert np.all(np.abs(g) <= s * (1 + 1e-15))
