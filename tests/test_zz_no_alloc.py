"""The allocation-free cubed-sphere stencil entry point.

Callers that cannot allocate device memory (a framework whose memory pool
forbids raw cudaMalloc, or code under a fixed device-memory budget) get the
cubed-sphere edge stencils from ``bc_cubed_sphere_stencils_noalloc``, which
keeps its scratch in a fixed device array inside the library.  Its rows must
agree with the ones the regular plan generates (``bc_plan_create`` with
``BC_GEOM_CUBED_SPHERE`` sub-matrices, read back through
``bc_plan_export_csr``) within the FP64 tolerance of the other tests, on two
calls in a row, and with the FP64 oracle's own geometry (``oracle.sphere``:
neighbour panel, depth row, stencil start and Lagrange weights, and the
basis change).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2605_14780_gb300 import bc, synth

TOL = 1e-12


def _plan_rows(N, h, p):
    """Rows of the regular plan, keyed by (panel, i, j, component)."""
    import torch
    w = synth.cubed_sphere(N, h, p, 1, ("h", "u", "v"), "f64", seed=21)
    ts = [torch.from_numpy(a.copy()).cuda() for a in w["fields"]]
    plan = bc.plan_for_workload(w, ts)
    ex = plan.export_csr()
    F = N + 2 * h
    rows = {}
    for r in range(len(ex["row_slot"])):
        slot = int(ex["row_slot"][r])
        panel, comp = divmod(slot, 3)
        off = int(ex["row_off"][r])
        i, j = off % F - h, off // F - h
        e0, e1 = ex["row_ptr"][r], ex["row_ptr"][r + 1]
        ents = [(divmod(int(ex["col_slot"][e]), 3),
                 int(ex["col_off"][e]) % F - h, int(ex["col_off"][e]) // F - h,
                 float(ex["val"][e])) for e in range(e0, e1)]
        rows[(panel, i, j, comp)] = ents
    return rows


def _cells(N, h):
    out = []
    for P in range(6):
        for strip in range(4):
            d, side = divmod(strip, 2)
            for r in range(h):
                for s in range(N):
                    g = N + r if side else -1 - r
                    out.append((P, g, s) if d == 0 else (P, s, g))
    return out


def _check_against_plan(res, rows, N, h, p):
    cells = _cells(N, h)
    assert len(cells) == len(res["nb"])
    for c, (P, i, j) in enumerate(cells):
        Q = int(res["nb"][c])
        i0, j0 = (int(x) for x in res["node0"][c])
        ax = int(res["axis"][c]) & 0xff
        snap = bool(int(res["axis"][c]) & bc.NOALLOC_SNAP)
        npts = 1 if snap else p
        nodes = [(i0 + k, j0) if ax == 0 else (i0, j0 + k) for k in range(npts)]
        wts = res["w"][c, :npts]
        # scalar component 0: entries (Q, comp 0, node_k, w_k)
        ents = rows[(P, i, j, 0)]
        assert [(e[0], e[1], e[2]) for e in ents] == [((Q, 0), n[0], n[1]) for n in nodes]
        assert np.allclose([e[3] for e in ents], wts, rtol=0, atol=TOL)
        # vector pair: u row = M00 w_k on Q.u, then M01 w_k on Q.v
        M = res["rot"][c]
        for comp, mrow in ((1, 0), (2, 1)):
            ents = rows[(P, i, j, comp)]
            exp = [((Q, 1), n[0], n[1], M[mrow, 0] * wk) for n, wk in zip(nodes, wts)] + \
                  [((Q, 2), n[0], n[1], M[mrow, 1] * wk) for n, wk in zip(nodes, wts)]
            assert [(e[0], e[1], e[2]) for e in ents] == [x[:3] for x in exp]
            assert np.allclose([e[3] for e in ents], [x[3] for x in exp], rtol=0, atol=TOL)


@pytest.mark.gpu
@pytest.mark.parametrize("N,h,p", [(13, 3, 6), (8, 2, 4)])
def test_noalloc_stencils_match_the_plan_twice(N, h, p):
    rows = _plan_rows(N, h, p)
    first = bc.cubed_sphere_stencils_noalloc(N, h, p, rotate=True)
    _check_against_plan(first, rows, N, h, p)
    second = bc.cubed_sphere_stencils_noalloc(N, h, p, rotate=True)
    _check_against_plan(second, rows, N, h, p)
    for k in first:
        assert np.array_equal(first[k], second[k])
    if N % 2 == 1:  # odd N: the centre line aligns and is copied
        assert np.any(first["axis"] & bc.NOALLOC_SNAP)


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_the_scratch():
    N = bc.NOALLOC_MAX_CELLS // (24 * 3) + 1
    with pytest.raises(bc.BCError) as e:
        bc.cubed_sphere_stencils_noalloc(N, 3, 6)
    assert e.value.status == "BC_ERR_UNSUPPORTED"
    assert "scratch" in str(e.value)
    with pytest.raises(bc.BCError) as e:
        bc.cubed_sphere_stencils_noalloc(4, 2, 6)
    assert e.value.status == "BC_ERR_INVALID_ARG"


@pytest.mark.gpu
@pytest.mark.parametrize("N,h,p", [(13, 3, 6), (8, 2, 4)])
def test_noalloc_stencils_match_the_oracle(N, h, p):
    """Every cell's neighbour panel, node-0 cell, stepping axis, snap flag,
    weights and basis change against the oracle's strip geometry."""
    from oracle import sphere
    res = bc.cubed_sphere_stencils_noalloc(N, h, p, rotate=True)
    c = 0
    for P in range(6):
        for d in range(2):
            for side in range(2):
                g = sphere.strip_geometry(P, N, h, d, side)
                snapped, start, w = sphere.stencil(g["t"], N, p)
                M = sphere.rotation(P, g["Q"], g["a"], g["b"], g["aq"], g["bq"])
                n = len(g["rq"])
                sl = slice(c, c + n)
                assert np.all(res["nb"][sl] == g["Q"])
                axis = res["axis"][sl]
                assert np.all((axis & 0xff) == 1 - g["dq"])
                assert np.array_equal((axis & bc.NOALLOC_SNAP) != 0, snapped)
                node = res["node0"][sl]
                assert np.array_equal(node[:, g["dq"]], g["rq"])
                assert np.array_equal(node[:, 1 - g["dq"]], start)
                wexp = np.where(snapped[:, None], np.eye(p)[0][None, :], w)
                assert np.allclose(res["w"][sl], wexp, rtol=0, atol=TOL)
                assert np.allclose(res["rot"][sl], M, rtol=0, atol=TOL)
                c += n
    assert c == 24 * N * h
