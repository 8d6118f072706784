"""Pins of the oracle's user interpolation-table rows (``Itp`` given by the
user, Sec. III-B) on the staggered two-block workload.

* a field that is a polynomial of degree < p along the edge is interpolated
  exactly to the staggered ghost positions (Lagrange reproduction);
* a constant covariant pair comes out turned by each ghost's own angle
  (the weights sum to one, then the 2x2 table applies);
* a transposed rotation table is caught by that closed form.
"""
import numpy as np
import pytest

from oracle import rows as oracle_rows
from oracle.operator import apply, build_operator
from paper_2605_14780_gb300 import synth


def _fill(w, fn):
    for blk, a in zip(w["blocks"], w["fields"]):
        d = synth.data_view(a, blk)
        n = blk["n"]
        jj, ii = np.meshgrid(np.arange(n[1]), np.arange(n[0]), indexing="ij")
        for c in range(a.shape[0]):
            for lev in range(a.shape[1]):
                d[c, lev, 0] = fn(c, lev, ii, jj)


@pytest.mark.parametrize("p", [2, 3, 4, 6])
def test_polynomials_along_the_edge_are_reproduced(p):
    nx, ny, h = 10, 14, 2
    w = synth.staggered_interp(nx=nx, ny=ny, h=h, p=p, rotate=False)
    coef = np.random.default_rng(p).normal(size=p)

    def poly(y):
        return sum(c * y ** k for k, c in enumerate(coef))
    _fill(w, lambda c, lev, i, j: poly(j) + 0.0 * i + lev)
    y = apply(build_operator(w), w["fields"])
    for b, shift in ((0, 0.5), (1, -0.5)):
        a = y[b][0]
        cols = range(h + nx, 2 * h + nx) if b == 0 else range(0, h)
        for lev in range(a.shape[0]):
            for col in cols:
                got = a[lev, 0, h:h + ny, col]
                want = poly(np.arange(ny) + shift) + lev
                assert np.allclose(got, want, rtol=0, atol=1e-10 * (1 + np.abs(want).max()))


def _turned_constant_error(w):
    U, V = 0.7, -1.3
    _fill(w, lambda c, lev, i, j: (0.0 * i + (U if c == 1 else V if c == 2 else 1.0)))
    y = apply(build_operator(w), w["fields"])
    nx, ny, h = w["blocks"][0]["n"][0], w["blocks"][0]["n"][1], w["blocks"][0]["h"][0]
    err = 0.0
    for b in (0, 1):
        for r in range(h):
            col = h + nx + r if b == 0 else h - 1 - r
            s = np.arange(ny)
            th = 0.05 * (s + 1) * (r + 1)
            u = y[b][1, 0, 0, h:h + ny, col]
            v = y[b][2, 0, 0, h:h + ny, col]
            err = max(err, float(np.max(np.abs(u - (np.cos(th) * U - np.sin(th) * V)))),
                      float(np.max(np.abs(v - (np.sin(th) * U + np.cos(th) * V)))))
    return err


def test_constant_pair_is_turned_by_each_ghosts_angle():
    assert _turned_constant_error(synth.staggered_interp()) < 1e-13


def test_pin_catches_transposed_rotation(monkeypatch):
    real = oracle_rows.interp_rows

    def transposed(bc):
        bc = dict(bc)
        bc["rot"] = np.asarray(bc["rot"]).reshape(-1, 2, 2).transpose(0, 2, 1).reshape(-1, 4)
        return real(bc)
    import oracle.operator as op_mod
    monkeypatch.setattr(op_mod, "interp_rows", transposed)
    assert _turned_constant_error(synth.staggered_interp()) > 1e-3


def test_axis_swap_transposes_the_result():
    """The workload with axes 0 and 1 exchanged (stencils stepping along
    axis 0) gives the transposed ghost values."""
    w = synth.staggered_interp(nx=10, ny=7, h=2, nlevels=2, p=4)
    v = synth.swap_xy(w)
    y = apply(build_operator(w), w["fields"])
    z = apply(build_operator(v), v["fields"])
    for a, b in zip(y, z):
        assert np.allclose(a.swapaxes(3, 4), b, rtol=0, atol=1e-13, equal_nan=True)
