"""Pins of the oracle's cubed-sphere interpolation rows.

* neighbour, depth row and along index against a brute-force nearest-cell
  search in 3-D (no use of the oracle's projection code);
* weights reproduce polynomials up to degree p-1 and sum to one;
* smooth scalar fields and covariant rigid-rotation winds synthesised by an
  independent finite-difference basis converge at O(Delta^p) (ratio >= 2^(p-1)
  per halving);
* the 2x2 basis change maps neighbour covariant components to own covariant
  components of arbitrary tangent vectors, with the bases taken by finite
  differences;
* adjacency is symmetric.
"""

import numpy as np
import pytest

from oracle import sphere
from oracle.operator import apply, build_operator
from paper_2605_14780_gb300 import synth


def _diag(N, h, p, fields=("scalar",), nlevels=1):
    w = synth.cubed_sphere(N, h, p, nlevels, fields, "f64", seed=1)
    diag = []
    op = build_operator(w, diagnostics=diag)
    return w, op, diag


@pytest.mark.parametrize("N,h", [(4, 1), (5, 2), (8, 3), (7, 3)])
def test_neighbour_by_brute_force(N, h):
    _, _, diag = _diag(N, h, min(4, N))
    # every data cell centre of every panel, by the generator's own geometry
    centres, ids = [], []
    ang = synth.cell_angle(N, np.arange(N))
    A, B = np.meshgrid(ang, ang, indexing="xy")     # [j, i]
    for P in range(6):
        X, Y, Z = synth._panel_xyz(P, A, B)
        centres.append(np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1))
        jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        ids.append(np.stack([np.full(N * N, P), ii.ravel(), jj.ravel()], 1))
    centres = np.concatenate(centres)
    ids = np.concatenate(ids)
    for d in diag:
        cells = d["cells"]
        a = synth.cell_angle(N, cells[:, 0])
        b = synth.cell_angle(N, cells[:, 1])
        X, Y, Z = synth._panel_xyz(d["P"], a, b)
        g = np.stack([X, Y, Z], 1)
        near = np.argmax(g @ centres.T, axis=1)     # nearest on the sphere
        q, qi, qj = ids[near].T
        assert np.all(q == d["Q"])
        qdepth = qi if d["dq"] == 0 else qj
        qalong = qi if d["dq"] == 1 else qj
        assert np.array_equal(qdepth, d["rq"])
        assert np.all(np.abs(qalong - np.rint(d["t"])) <= 1)


def test_adjacency_is_symmetric():
    _, _, diag = _diag(6, 2, 4)
    edge = {(d["P"], d["d"], d["side"]): (d["Q"], d["dq"], d["q_side"])
            for d in diag}
    assert len(edge) == 24
    for (P, dd, s), (Q, dq, qs) in edge.items():
        assert edge[(Q, dq, qs)] == (P, dd, s)
    # each panel meets four distinct panels, never itself or its antipode
    for P in range(6):
        nb = {edge[(P, dd, s)][0] for dd in (0, 1) for s in (0, 1)}
        assert len(nb) == 4 and P not in nb


@pytest.mark.parametrize("p", [2, 4, 6])
def test_weights_reproduce_polynomials(p):
    _, _, diag = _diag(12, 3, p)
    for d in diag:
        m = ~d["snapped"]
        t, st, w = d["t"][m], d["start"][m], d["w"][m]
        nodes = st[:, None] + np.arange(p)[None, :]
        for deg in range(p):
            lhs = np.sum(w * nodes.astype(np.float64) ** deg, axis=1)
            scale = np.sum(np.abs(w) * np.abs(nodes) ** deg, axis=1)
            assert np.all(np.abs(lhs - t ** deg) <= 1e-13 * scale + 1e-300)


def test_rows_sum_to_one_and_snaps_are_copies():
    w, op, diag = _diag(9, 2, 4)   # odd N: the centre line snaps
    assert sum(int(d["snapped"].sum()) for d in diag) == 24 * 2
    sums = np.asarray(op.A.sum(axis=1)).ravel()
    assert np.all(np.abs(sums - 1.0) < 1e-14)
    # snapped rows are single unit entries
    lay = op.layout
    for d in diag:
        for cell in d["cells"][d["snapped"]]:
            r = lay.row(np.array([d["P"]]), 0, 0, cell[None, :])[0]
            k = np.searchsorted(op.rows, r)
            row = op.A.getrow(k)
            assert row.nnz == 1 and row.data[0] == 1.0


def _smooth(X, Y, Z):
    return np.exp(0.7 * X - 0.3 * Y) * np.cos(1.3 * Z + 0.2) + X * Y * Z


def _scalar_error(N, p):
    h = 3
    w = synth.cubed_sphere(N, h, p, 1, ("scalar",), "f64", seed=1)
    ang_full = synth.cell_angle(N, np.arange(-h, N + h))
    A, B = np.meshgrid(ang_full, ang_full, indexing="xy")
    exact = []
    for P in range(6):
        X, Y, Z = synth._panel_xyz(P, A, B)
        exact.append(_smooth(X, Y, Z))
        d = synth.data_view(w["fields"][P], w["blocks"][P])
        d[0, 0, 0] = exact[P][h:h + N, h:h + N]
    y = apply(build_operator(w), w["fields"])
    err = 0.0
    for P in range(6):
        g = y[P][0, 0, 0]
        m = np.zeros_like(g, bool)
        m[h:h + N, :h] = m[h:h + N, N + h:] = True
        m[:h, h:h + N] = m[N + h:, h:h + N] = True
        err = max(err, float(np.max(np.abs(g[m] - exact[P][m]))))
    return err


@pytest.mark.parametrize("p", [4, 6])
def test_scalar_convergence(p):
    e = [_scalar_error(N, p) for N in (16, 32, 64)]
    assert e[0] / e[1] >= 2 ** (p - 1) and e[1] / e[2] >= 2 ** (p - 1), e


def _vector_error(N, p):
    h = 3
    axis = np.array([0.3, -0.5, 0.81])
    axis /= np.linalg.norm(axis)
    w = synth.cubed_sphere(N, h, p, 1, ("h", "u", "v"), "f64", seed=2)
    ang_full = synth.cell_angle(N, np.arange(-h, N + h))
    A, B = np.meshgrid(ang_full, ang_full, indexing="xy")
    exact = []
    for P in range(6):
        ua, ub = synth.rigid_rotation_covariant(P, A, B, axis, 50.0)
        exact.append((ua, ub))
        d = synth.data_view(w["fields"][P], w["blocks"][P])
        d[1, 0, 0] = ua[h:h + N, h:h + N]
        d[2, 0, 0] = ub[h:h + N, h:h + N]
    y = apply(build_operator(w), w["fields"])
    err = 0.0
    for P in range(6):
        m = np.zeros((N + 2 * h,) * 2, bool)
        m[h:h + N, :h] = m[h:h + N, N + h:] = True
        m[:h, h:h + N] = m[N + h:, h:h + N] = True
        for c in (1, 2):
            g = y[P][c, 0, 0]
            err = max(err, float(np.max(np.abs(g[m] - exact[P][c - 1][m]))))
    return err


@pytest.mark.parametrize("p", [4, 6])
def test_rigid_rotation_convergence(p):
    e = [_vector_error(N, p) for N in (16, 32, 64)]
    assert e[0] / e[1] >= 2 ** (p - 1) and e[1] / e[2] >= 2 ** (p - 1), e


def test_rotation_maps_covariant_components():
    """M (V . e_Q) == V . e_P for random tangent V, bases by central FD."""
    rng = np.random.default_rng(0)
    N, h = 10, 3
    for P in range(6):
        for dd in (0, 1):
            for side in (0, 1):
                g = sphere.strip_geometry(P, N, h, dd, side)
                M = sphere.rotation(P, g["Q"], g["a"], g["b"], g["aq"], g["bq"])
                for k in range(len(g["a"])):
                    axis = rng.normal(size=3)
                    axis /= np.linalg.norm(axis)
                    own = np.array(synth.rigid_rotation_covariant(
                        P, g["a"][k], g["b"][k], axis, 1.0))
                    nb = np.array(synth.rigid_rotation_covariant(
                        g["Q"], g["aq"][k], g["bq"][k], axis, 1.0))
                    assert np.allclose(M[k] @ nb, own, atol=2e-8, rtol=0)


def test_pin_catches_planted_weight_error(monkeypatch):
    """Dropping one factor of the Lagrange product breaks reproduction."""
    def bad(tau, p):
        tau = np.asarray(tau, np.float64).reshape(-1)
        w = np.ones((len(tau), p))
        for k in range(p):
            for m in range(p):
                if m != k and m != (k + 1) % p:
                    w[:, k] *= (tau - m) / (k - m)
        return w
    monkeypatch.setattr(sphere, "lagrange_weights", bad)
    _, _, diag = _diag(12, 3, 4)
    d = diag[0]
    m = ~d["snapped"]
    nodes = d["start"][m][:, None] + np.arange(4)[None, :]
    lhs = np.sum(d["w"][m] * nodes, axis=1)
    assert not np.allclose(lhs, d["t"][m])


def test_pin_catches_transposed_rotation(monkeypatch):
    real = sphere.rotation

    def bad(*a):
        return np.transpose(real(*a), (0, 2, 1))
    monkeypatch.setattr(sphere, "rotation", bad)
    e32 = _vector_error(32, 4)
    monkeypatch.setattr(sphere, "rotation", real)
    assert e32 > 100 * _vector_error(32, 4)
