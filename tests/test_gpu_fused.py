"""Boundary conditions fused with the following stencil (bc_apply_stencil):
the stencil of the ghost-filled field against the oracle's ghost fill
followed by the same stencil on the CPU, and the fields' covered ghosts
bit for bit as the oracle's copies and zero rows (within tolerance for
interpolation and CSR rows), for full and pruned plans."""
import numpy as np
import pytest

from gpu_util import TOL, compare, flat, to_device, to_device_innermost
from oracle.operator import apply, build_operator, row_scale
from paper_2605_14780_gb300 import bc, synth

pytestmark = pytest.mark.gpu

HPCG27 = (bc.box_stencil(3, 1),
          np.array([26.0 if tuple(o) == (0, 0, 0) else -1.0 for o in bc.box_stencil(3, 1)]))


def _reference(w, op, offsets, coeffs):
    """The stencil on the oracle's filled fields, and its error scale:
    the same stencil with |c| on |data| and, at covered ghosts, the row
    scale sum_e |a_e x_e| + |b|."""
    filled = apply(op, w["fields"])
    absf = [np.abs(a.astype(np.float64)) for a in w["fields"]]
    flat_abs = op.layout.flatten_full(absf)
    flat_abs[op.rows] = row_scale(op, w["fields"])
    absf = op.layout.unflatten_full(flat_abs, absf)
    outs, scales = [], []
    for f, af, blk in zip(filled, absf, w["blocks"]):
        n, h = blk["n"], blk["h"]
        o = np.zeros(f.shape)
        sc = np.zeros(f.shape)
        sl = (slice(h[2], h[2] + n[2]), slice(h[1], h[1] + n[1]), slice(h[0], h[0] + n[0]))
        for (di, dj, dk), c in zip(offsets, coeffs):
            src = (slice(h[2] + dk, h[2] + dk + n[2]), slice(h[1] + dj, h[1] + dj + n[1]),
                   slice(h[0] + di, h[0] + di + n[0]))
            o[(Ellipsis,) + sl] += c * f[(Ellipsis,) + src].astype(np.float64)
            sc[(Ellipsis,) + sl] += abs(c) * af[(Ellipsis,) + src]
        outs.append(o)
        scales.append(sc)
    return outs, scales


def _data_mask(w):
    ms = []
    for a, blk in zip(w["fields"], w["blocks"]):
        n, h = blk["n"], blk["h"]
        m = np.zeros(a.shape, bool)
        m[..., h[2]:h[2] + n[2], h[1]:h[1] + n[1], h[0]:h[0] + n[0]] = True
        ms.append(m)
    return ms


def _fused(w, offsets, coeffs, layout="outermost", pruned=False):
    import torch
    dev = to_device_innermost if layout == "innermost" else to_device
    ts = dev(w["fields"])
    outs = dev([np.zeros_like(a) for a in w["fields"]])
    plan = bc.plan_for_workload(w, ts, {"stencil_fusion": 1},
                                stencil=offsets if pruned else None)
    plan.apply_stencil(bc.slot_table(ts), bc.slot_table(outs), offsets, coeffs)
    torch.cuda.synchronize()
    return plan, [t.cpu().numpy() for t in ts], [o.cpu().numpy() for o in outs]


def _check(w, offsets, coeffs, fields, outs, op=None, pruned=False):
    op = op or build_operator(w)
    ref, scale = _reference(w, op, offsets, coeffs)
    tol = TOL[w["dtype"]] + len(coeffs) * (2.0 ** -24 if w["dtype"] == "f32" else 2.0 ** -53)
    for o, r, sc, m in zip(outs, ref, scale, _data_mask(w)):
        err = np.abs(o[m].astype(np.float64) - r[m])
        assert np.all(err <= tol * sc[m] + 1e-300), np.max(err / (tol * sc[m] + 1e-300))
        assert np.all(o[~m] == 0)  # ghosts of out untouched
    if not pruned:
        compare(w, fields, op=op)


@pytest.mark.parametrize("variant", ["Z", "P", "S"])
@pytest.mark.parametrize("n", [(6, 5, 7), (17, 9, 12)])
def test_hpcg_27_point(variant, n):
    w = synth.hpcg_block(n, variant, seed=41, nblocks=3)
    _, fields, outs = _fused(w, *HPCG27)
    _check(w, *HPCG27, fields, outs)


def test_hpcg_27_point_closed_form():
    """x = 1 everywhere: the 27-point output is 27 - prod_d c_d (c_d = 2 on
    a zero face, 3 otherwise) -- 0 inside, 9 on faces, 15 on edges, 19 on
    corners of the all-zero variant."""
    w = synth.hpcg_block((6, 6, 6), "Z", seed=1)
    for a in w["fields"]:
        a[np.isfinite(a)] = 1.0
    _, _, outs = _fused(w, *HPCG27)
    o = outs[0][0, 0, 1:-1, 1:-1, 1:-1]
    nb = np.zeros((6, 6, 6), int)
    for d in range(3):
        ax = np.arange(6)
        sh = [1, 1, 1]
        sh[2 - d] = 6
        nb += ((ax == 0) | (ax == 5)).reshape(sh)
    expect = np.choose(nb, [0.0, 9.0, 15.0, 19.0])
    assert np.array_equal(o, expect)


@pytest.mark.parametrize("layout", ["outermost", "innermost"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("pruned", [False, True])
def test_batching_box9(layout, dtype, pruned):
    """Uneven 2-D blocks (maps, zero, CSR edges) with a 9-point box stencil
    of random weights, full and pruned plans, both level layouts."""
    w = synth.batching(nblocks=30, side_lo=3, side_hi=40, lev_lo=1, lev_hi=12, h=2,
                       seed=42, dtype=dtype)
    offs = bc.box_stencil(2, 1)
    cf = np.random.default_rng(3).uniform(-1, 1, len(offs))
    _, fields, outs = _fused(w, offs, cf, layout, pruned)
    _check(w, offs, cf, fields, outs, pruned=pruned)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_cubed_sphere_star5(dtype):
    """Interpolated, rotated and CSR corner ghosts evaluated where a 5-point
    star stencil reads them (h = 2, a radius-2 star)."""
    w = synth.cubed_sphere(10, 2, 4, 3, ("h", "u", "v"), dtype, seed=43)
    offs = bc.star_stencil(2, 2)
    cf = np.random.default_rng(4).uniform(-1, 1, len(offs))
    _, fields, outs = _fused(w, offs, cf)
    _check(w, offs, cf, fields, outs)


def test_stencil_errors():
    import torch
    w = synth.hpcg_block((5, 5, 5), "P", seed=44)
    ts = to_device(w["fields"])
    outs = to_device([np.zeros_like(a) for a in w["fields"]])
    plain = bc.plan_for_workload(w, ts)
    with pytest.raises(bc.BCError) as e:
        plain.apply_stencil(bc.slot_table(ts), bc.slot_table(outs), *HPCG27)
    assert e.value.status == "BC_ERR_UNSUPPORTED"
    plan = bc.plan_for_workload(w, ts, {"stencil_fusion": 1})
    with pytest.raises(bc.BCError) as e:
        plan.apply_stencil(bc.slot_table(ts), bc.slot_table(outs), [(2, 0, 0)], [1.0])
    assert e.value.status == "BC_ERR_HALO_TOO_WIDE"
    with pytest.raises(bc.BCError) as e:
        plan.apply_stencil(bc.slot_table(ts), bc.slot_table(outs), [(0, 0, 0)], [np.nan])
    assert e.value.status == "BC_ERR_INVALID_ARG"
    torch.cuda.synchronize()


def test_hpcg_128_blocks_27_point():
    """The bench's fused workload at full size per block: 4 blocks of 128^3
    FP64 (x periodic), 27-point operator, every output against the CPU."""
    w = synth.hpcg_block(128, "P", seed=45, nblocks=4)
    _, fields, outs = _fused(w, *HPCG27)
    _check(w, *HPCG27, fields, outs)
