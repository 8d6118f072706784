"""Oracle pins of block-edge averaging (``Sync``, Sec. III-B) and of the
in-place adjoint: closed forms on the shared nodes, constants preserved, and
``apply_adjoint`` equal to the transpose of a Jacobian built column by column
from ``apply`` (brute force, tiny grids)."""
import numpy as np
import pytest

from oracle.operator import OracleError, apply, apply_adjoint, build_operator
from paper_2605_14780_gb300 import synth


def _copies(w, n, bx, by):
    """Physical node -> list of (block, i, j) copies, from the block layout."""
    out = {}
    for b in range(by):
        for a in range(bx):
            for j in range(n):
                for i in range(n):
                    out.setdefault((a * (n - 1) + i, b * (n - 1) + j), []).append(
                        (b * bx + a, i, j))
    return out


def test_shared_nodes_become_the_mean_of_their_copies():
    bx, by, n, h = 3, 2, 6, 2
    w = synth.sync_grid(bx, by, n, h, nlevels=3, ncomp=2, dtype="f64", seed=3)
    out = apply(build_operator(w), w["fields"])
    for grp in _copies(w, n, bx, by).values():
        for c in range(2):
            for lev in range(3):
                vin = [w["fields"][b][c, lev, 0, h + j, h + i] for b, i, j in grp]
                vout = [out[b][c, lev, 0, h + j, h + i] for b, i, j in grp]
                if len(grp) == 1:
                    assert vout[0] == vin[0]
                else:
                    assert np.allclose(vout, np.mean(vin), rtol=0, atol=1e-15)


def test_ghosts_read_the_values_before_averaging():
    """One application of A: the halo ghost at depth 0 right of block 0 is
    the right neighbour's node 1 as it was on input."""
    n, h = 6, 2
    w = synth.sync_grid(2, 1, n, h, nlevels=1, ncomp=1, dtype="f64", seed=4)
    out = apply(build_operator(w), w["fields"])
    for j in range(n):
        assert out[0][0, 0, 0, h + j, h + n] == w["fields"][1][0, 0, 0, h + j, h + 1]


def test_constants_are_preserved():
    w = synth.sync_grid(3, 3, 5, 1, nlevels=2, ncomp=1, dtype="f64", seed=5)
    for a, blk in zip(w["fields"], w["blocks"]):
        a[...] = 7.0
    out = apply(build_operator(w), w["fields"])
    for a in out:
        v = a[0, :, 0, 1:-1, 1:-1]
        assert np.all(v == 7.0)


def _jacobian(w):
    """Columns J e_k of the affine in-place map, k over every stored value."""
    sizes = [a.size for a in w["fields"]]
    N = sum(sizes)
    op = build_operator(w)

    def f(vec):
        fields, k = [], 0
        for a in w["fields"]:
            fields.append(vec[k:k + a.size].reshape(a.shape))
            k += a.size
        return np.concatenate([x.ravel() for x in apply(op, fields)])

    base = f(np.zeros(N))
    J = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        J[:, k] = f(e) - base
    return op, J


@pytest.mark.parametrize("make", [
    lambda: synth.sync_grid(2, 2, 4, 1, nlevels=2, ncomp=1, dtype="f64", seed=6),
    lambda: synth.alg1_example(dtype="f64"),
])
def test_adjoint_is_the_transpose_of_the_brute_force_jacobian(make):
    w = make()
    for a in w["fields"]:
        a[np.isnan(a)] = 0.0
    op, J = _jacobian(w)
    rng = np.random.default_rng(8)
    ybar = [rng.uniform(-1, 1, a.shape) for a in w["fields"]]
    got = np.concatenate([x.ravel() for x in apply_adjoint(op, ybar)])
    ref = J.T @ np.concatenate([y.ravel() for y in ybar])
    assert np.allclose(got, ref, rtol=0, atol=1e-14)


def test_sync_rows_must_be_data_cells():
    w = synth.sync_grid(2, 1, 5, 1, nlevels=1, ncomp=1, dtype="f64", seed=9)
    s = next(b for b in w["bcs"] if b["kind"] == "sync")
    s["lo"] = (-1, s["lo"][1], 0)
    s["hi"] = (0, s["hi"][1], 1)
    with pytest.raises(OracleError):
        build_operator(w)


def test_two_level_injection_and_prolongation():
    """Region steps 1 and 2 (Sec. III-A): the coarse block's left ghosts are
    the fine cells at the lower-left corner of each coarse cell, the fine
    block's right ghosts the coarse cells containing them."""
    nx, ny, h = 12, 8, 2
    w = synth.two_level(nx, ny, h, nlevels=2, ncomp=2, dtype="f64", seed=3)
    out = apply(build_operator(w), w["fields"])
    f, c = w["fields"][0], w["fields"][1]
    for r in range(h):
        for j in range(ny // 2):
            # coarse ghost i = -1 - r  <-  fine data x = nx - 2 - 2 r, y = 2 j
            assert np.array_equal(out[1][:, :, 0, h + j, h - 1 - r],
                                  f[:, :, 0, h + 2 * j, h + nx - 2 - 2 * r])
        for j in range(ny):
            # fine ghost i = nx + r  <-  coarse data (r // 2, j // 2)
            assert np.array_equal(out[0][:, :, 0, h + j, h + nx + r],
                                  c[:, :, 0, h + j // 2, h + r // 2])
