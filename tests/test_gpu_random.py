"""Seeded random sweep: many small workloads of every description type, in
both level layouts and all launch forms, forward and adjoint against the
oracle.  Each case is small enough for the oracle to build in well under a
second."""
import numpy as np
import pytest

from gpu_util import TOL, compare, flat, run, to_device, to_device_innermost
from oracle.operator import apply_adjoint, build_operator
from paper_2605_14780_gb300 import bc, synth

pytestmark = pytest.mark.gpu


def _random_workload(seed):
    rng = np.random.default_rng(seed)
    kind = seed % 5
    dtype = ("f32", "f64")[int(rng.integers(2))]
    if kind == 0 or kind == 1:
        h = int(rng.integers(1, 4))
        return synth.batching(nblocks=int(rng.integers(1, 24)), side_lo=h, side_hi=int(rng.integers(h, 40)),
                              lev_lo=1, lev_hi=int(rng.integers(1, 40)), h=h, seed=seed, dtype=dtype)
    if kind == 2:
        N = int(rng.integers(4, 14))
        h = int(rng.integers(1, min(3, N // 2) + 1))
        p = int(rng.choice([2, 4, 6][: 1 + (N >= 6) + (N >= 8)]))
        return synth.cubed_sphere(N, h, p, int(rng.integers(1, 6)), ("h", "u", "v"), dtype,
                                  seed=seed)
    if kind == 3:
        return synth.sync_grid(int(rng.integers(1, 4)), int(rng.integers(1, 4)),
                               int(rng.integers(3, 9)), int(rng.integers(1, 3)),
                               int(rng.integers(1, 6)), int(rng.integers(1, 3)), dtype, seed=seed)
    nx = 2 * int(rng.integers(2, 12))
    ny = 2 * int(rng.integers(2, 10))
    return synth.two_level(nx, ny, int(rng.integers(1, 3)), int(rng.integers(1, 5)),
                           int(rng.integers(1, 3)), dtype, seed=seed)


@pytest.mark.parametrize("seed", range(40))
def test_random_forward(seed):
    import torch
    w = _random_workload(seed)
    rng = np.random.default_rng(1000 + seed)
    layout = int(rng.integers(2))
    form = [bc.BC_FORM_BATCHED, bc.BC_FORM_TYPEWIDE, bc.BC_FORM_PER_BC][int(rng.integers(3))]
    opts = {"units_per_lane": int(rng.choice([1, 2, 4, 8])),
            "threads": int(rng.choice([64, 128, 256])),
            "no_runs": int(rng.integers(2))}
    ts = to_device_innermost(w["fields"]) if layout else to_device(w["fields"])
    run(w, form=form, opts=opts, tensors=ts)
    torch.cuda.synchronize()
    compare(w, [t.cpu().numpy() for t in ts])


@pytest.mark.parametrize("seed", range(0, 40, 3))
def test_random_adjoint(seed):
    import torch
    w = _random_workload(seed)
    layout = seed % 2
    dev = to_device_innermost if layout else to_device
    ts = dev(w["fields"])
    plan = bc.plan_for_workload(w, ts)
    cot = synth.cotangent_like(w, 500 + seed)
    cs = dev(cot)
    plan.adjoint(bc.slot_table(cs))
    torch.cuda.synchronize()
    got = flat([c.cpu().numpy() for c in cs]).astype(np.float64)
    op = build_operator(w)
    ref = flat(apply_adjoint(op, cot))
    y = flat(cot).astype(np.float64)
    scale = np.abs(y).copy()
    scale[op.layout.data_rows()] += abs(op.A).T @ np.abs(y[op.rows])
    assert np.all(np.abs(got - ref) <= TOL[w["dtype"]] * scale)


def _random_quadrature(seed):
    rng = np.random.default_rng(seed)
    N = int(rng.integers(4, 15))
    h = int(rng.integers(1, min(3, N // 2) + 1))
    p = int(rng.integers(2, min(8, N) + 1))
    nq = int(rng.integers(1, 5))
    fields = (("scalar",), ("h", "u", "v"))[int(rng.integers(2))]
    dtype = ("f32", "f64")[int(rng.integers(2))]
    return synth.cubed_sphere(N, h, p, int(rng.integers(1, 7)), fields, dtype, seed=seed,
                              quad=nq)


@pytest.mark.parametrize("seed", range(12))
def test_random_quadrature(seed):
    """Reconstruction-and-quadrature rows of random order, Gauss points,
    halo, levels, layout, launch form and item shape: forward and adjoint."""
    import torch
    w = _random_quadrature(300 + seed)
    rng = np.random.default_rng(2000 + seed)
    layout = int(rng.integers(2))
    form = [bc.BC_FORM_BATCHED, bc.BC_FORM_TYPEWIDE, bc.BC_FORM_PER_BC][int(rng.integers(3))]
    opts = {"units_per_lane": int(rng.choice([1, 2, 4, 8])),
            "threads": int(rng.choice([64, 128, 256]))}
    dev = to_device_innermost if layout else to_device
    ts = dev(w["fields"])
    plan, _ = run(w, form=form, opts=opts, tensors=ts)
    compare(w, [t.cpu().numpy() for t in ts])
    cot = synth.cotangent_like(w, 700 + seed)
    cs = dev(cot)
    plan.adjoint(bc.slot_table(cs))
    torch.cuda.synchronize()
    got = flat([c.cpu().numpy() for c in cs]).astype(np.float64)
    op = build_operator(w)
    ref = flat(apply_adjoint(op, cot))
    y = flat(cot).astype(np.float64)
    scale = np.abs(y).copy()
    scale[op.layout.data_rows()] += abs(op.A).T @ np.abs(y[op.rows])
    assert np.all(np.abs(got - ref) <= TOL[w["dtype"]] * scale)
