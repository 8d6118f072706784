"""Pins of the oracle's reconstruction-and-quadrature cubed-sphere rows
(the finite-volume form of the HOPE example, Sec. II-B; ``Itp = Agg . Recons``,
Sec. III-B).

* the one-dimensional reconstruction from cell averages against closed forms
  (linear and quadratic) and exactly on random polynomials of degree < p, the
  averages integrated by exact antiderivatives;
* scalar rows sum to one and hold p^2 entries (2 p^2 for a vector pair);
* data set to exact cell averages of a smooth field (dense Gauss rule on the
  generator's own panel geometry) give ghost values that converge to the
  exact ghost-cell averages at O(Delta^min(p, 2 nq));
* covariant rigid-rotation winds (basis by finite differences in the
  generator) converge the same way;
* planted mistakes in the oracle (point interpolation instead of
  reconstruction from averages, a transposed rotation) break the pins.
"""
import math

import numpy as np
import pytest

from oracle import sphere
from oracle.operator import apply, build_operator
from paper_2605_14780_gb300 import synth


def _antiderivative_averages(coef, p):
    """Averages over [k - 1/2, k + 1/2], k < p, of the polynomial ``coef``."""
    P = np.polynomial.Polynomial(coef).integ()
    k = np.arange(p, dtype=np.float64)
    return P(k + 0.5) - P(k - 0.5)


def test_reconstruction_closed_forms():
    rng = np.random.default_rng(0)
    x = rng.uniform(-1.0, 3.0, size=17)
    a = rng.normal(size=3)
    # two cells: the linear function through the averages (= centre values)
    c2 = sphere.average_reconstruction_weights(x, 2)
    assert np.allclose(c2 @ a[:2], a[0] + (a[1] - a[0]) * x, atol=1e-14, rtol=0)
    # three cells centred at 0, 1, 2: P(y) = b - s/24 + (c - a)/2 y + s/2 y^2,
    # y = x - 1, s = a - 2b + c
    c3 = sphere.average_reconstruction_weights(x, 3)
    y = x - 1.0
    s = a[0] - 2 * a[1] + a[2]
    ref = a[1] - s / 24 + (a[2] - a[0]) / 2 * y + s / 2 * y ** 2
    assert np.allclose(c3 @ a, ref, atol=1e-13, rtol=0)


@pytest.mark.parametrize("p", range(2, 9))
def test_reconstruction_exact_below_degree_p(p):
    rng = np.random.default_rng(p)
    x = rng.uniform(-0.5, p - 0.5, size=23)
    c = sphere.average_reconstruction_weights(x, p)
    assert np.allclose(c.sum(axis=1), 1.0, atol=1e-12, rtol=0)
    for deg in range(p):
        coef = rng.normal(size=deg + 1)
        got = c @ _antiderivative_averages(coef, p)
        ref = np.polynomial.Polynomial(coef)(x)
        assert np.allclose(got, ref, atol=1e-9 * (1 + np.abs(ref).max()), rtol=0), (p, deg)
    # degree p is not reproduced (the pin is not vacuous)
    coef = np.zeros(p + 1)
    coef[p] = 1.0
    assert not np.allclose(c @ _antiderivative_averages(coef, p),
                           np.polynomial.Polynomial(coef)(x), atol=1e-6)


@pytest.mark.parametrize("N,h,p,nq", [(8, 2, 4, 2), (9, 3, 3, 1), (10, 1, 6, 3), (6, 2, 2, 4)])
def test_rows_sum_to_one_with_full_patches(N, h, p, nq):
    w = synth.cubed_sphere(N, h, p, 1, ("h", "u", "v"), "f64", seed=4, quad=nq)
    op = build_operator(w)
    lay = op.layout
    rows_nnz = np.diff(op.A.indptr)
    sums = np.asarray(op.A.sum(axis=1)).ravel()
    b = np.searchsorted(lay.full_base, op.rows, side="right") - 1
    plane = lay.F.prod(axis=1) * lay.L
    comp = (op.rows - lay.full_base[b]) // plane[b]
    # edge rows: scalar rows p^2 entries summing to one, vector rows 2 p^2
    edge = rows_nnz >= p * p
    assert np.all(rows_nnz[edge & (comp == 0)] == p * p)
    assert np.allclose(sums[edge & (comp == 0)], 1.0, atol=1e-12, rtol=0)
    assert np.all(rows_nnz[edge & (comp > 0)] == 2 * p * p)
    assert edge.sum() == 6 * 4 * h * N * 3


def _cell_averages(P, N, ia, ib, fn, n=6):
    """Averages over cells (ia, ib) of panel ``P`` in its angle coordinates,
    by an ``n x n`` Gauss rule on the generator's geometry."""
    xg, wg = np.polynomial.legendre.leggauss(n)
    d = math.pi / (2 * N)
    a0 = synth.cell_angle(N, ia)
    b0 = synth.cell_angle(N, ib)
    acc = None
    for i in range(n):
        for j in range(n):
            v = fn(P, a0 + xg[i] * d / 2, b0 + xg[j] * d / 2)
            v = [wg[i] * wg[j] / 4 * t for t in v]
            acc = v if acc is None else [s + t for s, t in zip(acc, v)]
    return acc


def _smooth(P, a, b):
    X, Y, Z = synth._panel_xyz(P, a, b)
    return [np.exp(0.7 * X - 0.3 * Y) * np.cos(1.3 * Z + 0.2) + X * Y * Z]


_AXIS = np.array([0.3, -0.5, 0.81]) / np.linalg.norm([0.3, -0.5, 0.81])


def _wind(P, a, b):
    return list(synth.rigid_rotation_covariant(P, a, b, _AXIS, 50.0))


def _edge_mask(N, h):
    m = np.zeros((N + 2 * h,) * 2, bool)
    m[h:h + N, :h] = m[h:h + N, N + h:] = True
    m[:h, h:h + N] = m[N + h:, h:h + N] = True
    return m


def _quad_error(N, p, nq, vector):
    h = 2
    fields = ("h", "u", "v") if vector else ("scalar",)
    w = synth.cubed_sphere(N, h, p, 1, fields, "f64", seed=1, quad=nq)
    idx = np.arange(-h, N + h)
    I, J = np.meshgrid(idx, idx, indexing="xy")     # [j, i]
    fn = _wind if vector else _smooth
    comps = (1, 2) if vector else (0,)
    exact = []
    for P in range(6):
        avg = _cell_averages(P, N, I, J, fn)
        exact.append(avg)
        d = synth.data_view(w["fields"][P], w["blocks"][P])
        for c, v in zip(comps, avg):
            d[c, 0, 0] = v[h:h + N, h:h + N]
    y = apply(build_operator(w), w["fields"])
    m = _edge_mask(N, h)
    err = 0.0
    for P in range(6):
        for c, v in zip(comps, exact[P]):
            err = max(err, float(np.max(np.abs(y[P][c, 0, 0][m] - v[m]))))
    return err


@pytest.mark.parametrize("p,nq,Ns", [(2, 1, (16, 32)), (4, 2, (16, 32)), (3, 2, (16, 32)),
                                     (6, 3, (24, 48))])
def test_scalar_averages_converge(p, nq, Ns):
    order = min(p, 2 * nq)
    e = [_quad_error(N, p, nq, False) for N in Ns]
    assert math.log2(e[0] / e[1]) >= order - 0.7, (e, order)


def test_covariant_wind_averages_converge():
    e = [_quad_error(N, 4, 2, True) for N in (16, 32)]
    assert math.log2(e[0] / e[1]) >= 4 - 0.7, e
    assert e[1] < 1e-3 * 50.0


def test_pin_catches_point_interpolation(monkeypatch):
    """Treating the averages as centre values (Lagrange through the centres)
    costs two orders: the convergence pin fails."""
    def lagrange(x, p):
        return sphere.lagrange_weights(x, p)
    monkeypatch.setattr(sphere, "average_reconstruction_weights", lagrange)
    e = [_quad_error(N, 4, 2, False) for N in (16, 32)]
    assert math.log2(e[0] / e[1]) < 4 - 0.7


def test_pin_catches_transposed_rotation(monkeypatch):
    good = _quad_error(16, 4, 2, True)
    real = sphere.rotation
    monkeypatch.setattr(sphere, "rotation", lambda *a: np.transpose(real(*a), (0, 2, 1)))
    assert _quad_error(16, 4, 2, True) > 100 * good


def _mid_edge_error(N, p, nq, centred, sweeps):
    """Largest error over the middle half of every edge strip (away from the
    panel corners, whose CSR rows are only first-order)."""
    h = 3
    w = synth.cubed_sphere(N, h, p, 1, ("scalar",), "f64", seed=1, quad=nq, centred=centred,
                           sweeps=sweeps)
    idx = np.arange(-h, N + h)
    I, J = np.meshgrid(idx, idx, indexing="xy")
    exact = []
    for P in range(6):
        avg = _cell_averages(P, N, I, J, _smooth)[0]
        exact.append(avg)
        synth.data_view(w["fields"][P], w["blocks"][P])[0, 0, 0] = avg[h:h + N, h:h + N]
    y = apply(build_operator(w), w["fields"])
    q = N // 4
    m = np.zeros((N + 2 * h,) * 2, bool)
    m[h + q:h + N - q, :h] = m[h + q:h + N - q, N + h:] = True
    m[:h, h + q:h + N - q] = m[N + h:, h + q:h + N - q] = True
    return max(float(np.max(np.abs(y[P][0, 0, 0][m] - exact[P][m]))) for P in range(6))


def test_centred_patches_fold_to_a_converged_fixed_point():
    """Centred patches read the neighbour's ghost cells (HOPE(I)); the
    Jacobi sweeps have converged by ten (twenty change nothing), and one
    sweep (ghost columns dropped) is a different, worse answer."""
    ops = {}
    w = synth.cubed_sphere(12, 3, 4, 1, ("h", "u", "v"), "f64", seed=2, quad=2, centred=True)
    for k in (1, 10, 20):
        ops[k] = apply(build_operator(dict(w, ghost_sweeps=k)), w["fields"])
    diff = max(float(np.max(np.abs(a - b))) for a, b in zip(ops[10], ops[20]))
    first = max(float(np.max(np.abs(a - b))) for a, b in zip(ops[1], ops[10]))
    assert diff < 1e-9 * 1e4 and first > 1e-3


def test_centred_patches_converge_away_from_corners():
    e = [_mid_edge_error(N, 4, 2, True, 10) for N in (16, 32)]
    assert math.log2(e[0] / e[1]) >= 4 - 0.7, e
