"""GPU adjoint (A^T) against the oracle's explicit transpose, FP64 central
finite differences of the GPU forward, the dot-product test, and the
autograd Function."""
import numpy as np
import pytest

from gpu_util import TOL, bits, flat, run, to_device
from oracle.operator import apply_adjoint, build_operator
from paper_2605_14780_gb300 import bc, synth

pytestmark = pytest.mark.gpu


def _adjoint_gpu(w, cot, opts=None):
    import torch
    ts = to_device(w["fields"])
    plan = bc.plan_for_workload(w, ts, opts)
    cs = to_device(cot)
    plan.adjoint(bc.slot_table(cs))
    torch.cuda.synchronize()
    return plan, [c.cpu().numpy() for c in cs]


def _check_adjoint(w, cot, out, levels=None, op=None):
    """Data values: |gpu - oracle| <= tol * (|y_j| + sum_i |A_ij y_i|);
    covered ghosts exactly 0; uncovered ghosts and untouched data equal to
    the cotangent bit for bit."""
    op = op or build_operator(w, levels=levels)
    ref = flat(apply_adjoint(op, cot))
    got = flat(out).astype(np.float64)
    y = flat(cot).astype(np.float64)
    tol = TOL[w["dtype"]]
    g = np.abs(y[op.rows])
    scale = np.abs(y).copy()
    scale[op.layout.data_rows()] += abs(op.A).T @ g
    covered = np.zeros(y.size, bool)
    covered[op.rows] = True
    if levels is None:
        assert np.all(got[covered] == 0.0)
        chk = ~covered
    else:
        # only the sampled levels are exact in `ref`; compare their data rows
        chk = np.zeros(y.size, bool)
        dr = op.layout.data_rows()
        touched = np.zeros(op.layout.n_data, bool)
        touched[np.unique(op.A.indices)] = True
        chk[dr[touched]] = True
        chk &= _level_mask(w, levels)
    err = np.abs(got[chk] - ref[chk])
    assert np.all(err <= tol * scale[chk] + 0.0), np.max(err / (tol * scale[chk] + 1e-300))


def _level_mask(w, levels):
    parts = []
    for a in w["fields"]:
        m = np.zeros(a.shape, bool)
        m[:, [lv for lv in levels if lv < a.shape[1]]] = True
        parts.append(m.ravel())
    return np.concatenate(parts)


@pytest.mark.parametrize("make", [
    lambda: synth.alg1_example(dtype="f64"),
    lambda: synth.hpcg_block((7, 5, 6), "S", seed=3),
    lambda: synth.hpcg_block((7, 5, 6), "P", seed=3, dtype="f32"),
    lambda: synth.batching(nblocks=40, side_lo=3, side_hi=30, lev_lo=1,
                           lev_hi=19, h=2, seed=2, dtype="f32"),
    lambda: synth.cubed_sphere(9, 3, 6, 3, ("h", "u", "v"), "f64", seed=4),
    lambda: synth.cubed_sphere(16, 3, 6, 10, ("h", "u", "v"), "f32", seed=4),
    lambda: synth.two_level(20, 14, 2, nlevels=3, ncomp=2, dtype="f64", seed=5),
    lambda: synth.staggered_interp(nlevels=4, p=4, dtype="f64"),
    lambda: synth.staggered_interp(nlevels=9, p=6, dtype="f32"),
    lambda: synth.ghost_on_ghost(scheme="smooth", sweeps=5, dtype="f64"),
    lambda: synth.ghost_on_ghost(scheme="extrapolate", sweeps=3, dtype="f32", nlevels=4),
    lambda: synth.cubed_sphere(9, 3, 4, 3, ("h", "u", "v"), "f64", seed=4, quad=2),
    lambda: synth.cubed_sphere(8, 3, 4, 3, ("h", "u", "v"), "f64", seed=4, quad=2,
                               centred=True, sweeps=10),
    lambda: synth.cubed_sphere(14, 2, 6, 6, ("h", "u", "v"), "f32", seed=4, quad=3),
])
def test_adjoint_vs_oracle(make):
    w = make()
    cot = synth.cotangent_like(w, 77)
    _, out = _adjoint_gpu(w, cot)
    _check_adjoint(w, cot, out)


@pytest.mark.parametrize("make", [
    lambda: synth.batching(nblocks=30, side_lo=3, side_hi=30, lev_lo=1,
                           lev_hi=20, h=2, seed=3, dtype="f32"),
    lambda: synth.cubed_sphere(10, 3, 6, 9, ("h", "u", "v"), "f64", seed=4),
    lambda: synth.cubed_sphere(8, 2, 4, 7, ("h", "u", "v"), "f32", seed=4, quad=2),
])
def test_adjoint_level_innermost(make):
    import torch
    from gpu_util import to_device_innermost
    w = make()
    cot = synth.cotangent_like(w, 78)
    ts = to_device_innermost(w["fields"])
    plan = bc.plan_for_workload(w, ts)
    cs = to_device_innermost(cot)
    plan.adjoint(bc.slot_table(cs))
    torch.cuda.synchronize()
    _check_adjoint(w, cot, [c.cpu().numpy() for c in cs])


def test_adjoint_full_768_sampled():
    """The 6 x 768^2, (h, u, v) x 32-level FP32 adjoint, levels 2 and 29
    compared with the oracle's explicit transpose."""
    w = synth.adjoint_cubed_sphere()
    cot = synth.cotangent_like(w, 5)
    _, out = _adjoint_gpu(w, cot)
    _check_adjoint(w, cot, out, levels=[2, 29])


def test_sync_grid_bench_size_sampled():
    """The bench's block-edge averaging workload (8 x 8 blocks of 129^2
    nodes, h = 3, 3 components x 32 levels FP32): forward and adjoint,
    levels 0 and 31 against the oracle."""
    from gpu_util import compare
    w = synth.sync_grid(8, 8, 129, 3, 32, 3, "f32", seed=12)
    _, out = run(w)
    compare(w, out, levels=[0, 31])
    cot = synth.cotangent_like(w, 12)
    _, adj = _adjoint_gpu(w, cot)
    _check_adjoint(w, cot, adj, levels=[0, 31])


def test_hope_adjoint_sampled():
    """The 6 x 384^2 reconstruction-and-quadrature workload's adjoint (as the
    bench times it), levels 3 and 30 against the oracle's transpose."""
    w = synth.hope_cubed_sphere()
    cot = synth.cotangent_like(w, 31)
    _, out = _adjoint_gpu(w, cot)
    _check_adjoint(w, cot, out, levels=[3, 30])


def _fd_setup(N=10, L=3):
    w = synth.cubed_sphere(N, 3, 6, L, ("h", "u", "v"), "f64", seed=6)
    for a in w["fields"]:
        a[np.isnan(a)] = 0.0
    return w


def test_adjoint_central_fd_64_directions():
    """x_bar . d == y_bar . (F(x + e d) - F(x - e d)) / 2e with the GPU
    forward in FP64, 64 random data directions (exact for an affine map up to
    rounding)."""
    import torch
    w = _fd_setup()
    rng = np.random.default_rng(6)
    cot = synth.cotangent_like(w, 66)
    _, xbar = _adjoint_gpu(w, cot)
    xbar = flat(xbar)
    ts = to_device(w["fields"])
    plan = bc.plan_for_workload(w, ts)
    y = flat(cot).astype(np.float64)
    mask = [np.zeros(a.shape, bool) for a in w["fields"]]
    for m, blk in zip(mask, w["blocks"]):
        n, h = blk["n"], blk["h"]
        m[:, :, h[2]:h[2] + n[2], h[1]:h[1] + n[1], h[0]:h[0] + n[0]] = True
    eps = 0.25
    for _ in range(64):
        dirs = [np.where(m, rng.uniform(-1, 1, m.shape), 0.0) for m in mask]
        outs = []
        for sgn in (1.0, -1.0):
            xs = [torch.from_numpy(a + sgn * eps * d).cuda() for a, d in zip(w["fields"], dirs)]
            plan.apply(bc.slot_table(xs))
            torch.cuda.synchronize()
            outs.append(flat([x.cpu().numpy() for x in xs]))
        jd = (outs[0] - outs[1]) / (2 * eps)
        lhs = np.dot(y, jd)
        rhs = np.dot(xbar, flat(dirs))
        mag = np.sum(np.abs(y * jd)) + np.sum(np.abs(xbar * flat(dirs)))
        assert abs(lhs - rhs) <= 1e-13 * mag


def test_dot_product_identity_gpu():
    """<A x, y> == <x, A^T y> with both sides from the GPU (FP64),
    compensated sums, relative 1e-13."""
    import math
    w = _fd_setup(12, 4)
    rng = np.random.default_rng(1)
    for a in w["fields"]:
        a[...] = np.where(np.isnan(a), 0.0, a)
    _, fx = run(w)
    op = build_operator(w)
    covered = np.zeros(sum(a.size for a in w["fields"]), bool)
    covered[op.rows] = True
    ax = flat(fx)[covered]
    ycot = [rng.uniform(-1, 1, a.shape) for a in w["fields"]]
    yv = flat(ycot)
    ymask = np.where(covered, yv, 0.0)
    ycot_g = [c for c in op.layout.unflatten_full(ymask, w["fields"])]
    _, atyf = _adjoint_gpu(w, ycot_g)
    aty = flat(atyf)
    xd = np.zeros_like(aty)
    dr = op.layout.data_rows()
    xd[dr] = op.layout.data_vector(w["fields"])
    lhs = math.fsum((ax * yv[covered]).tolist())
    rhs = math.fsum((xd * aty).tolist())
    mag = math.fsum(np.abs(ax * yv[covered]).tolist())
    assert abs(lhs - rhs) <= 1e-13 * mag


def test_autograd_function():
    import torch
    w = synth.cubed_sphere(8, 2, 4, 2, ("h", "u", "v"), "f64", seed=8)
    for a in w["fields"]:
        a[np.isnan(a)] = 0.0
    ts = [t.requires_grad_(False) for t in to_device(w["fields"])]
    plan = bc.plan_for_workload(w, ts)
    leaves = [t.clone().requires_grad_(True) for t in ts]
    xs = [l * 1.0 for l in leaves]
    ys = bc.BCFill.apply(plan, *xs)
    cot = synth.cotangent_like(w, 9)
    loss = sum((y * torch.from_numpy(c).cuda()).sum() for y, c in zip(ys, cot))
    loss.backward()
    got = flat([l.grad.cpu().numpy() for l in leaves])
    ref = flat(apply_adjoint(build_operator(w), cot))
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    # the forward result is the ghost-filled field
    out = flat([y.detach().cpu().numpy() for y in ys])
    _, fwd = run(w)
    assert np.array_equal(bits(out), bits(flat(fwd)))


def _autograd(w, ts, cot):
    """Forward and backward of ``BCFill`` on fields ``ts`` (any layout the
    plan is built for): returns the plan, the ghost-filled fields and the
    leaves' gradients as host arrays in (C, L, F2, F1, F0) index order."""
    import torch
    leaves = [t.detach().clone().requires_grad_(True) for t in ts]
    xs = [l.clone() for l in leaves]  # keeps each leaf's strides
    plan = bc.plan_for_workload(w, xs)
    ys = bc.BCFill.apply(plan, *xs)
    loss = sum((y * torch.from_numpy(np.ascontiguousarray(c)).cuda()).sum()
               for y, c in zip(ys, cot))
    loss.backward()
    torch.cuda.synchronize()
    fwd = [y.detach().cpu().numpy() for y in ys]
    grads = [l.grad.cpu().numpy() for l in leaves]
    return plan, fwd, grads


@pytest.mark.parametrize("layout", ["level_outermost", "level_innermost"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_autograd_layouts(layout, dtype):
    """BCFill forward and backward on fields stored levels outermost and
    levels innermost (the plan reads the cotangents with the forward fields'
    strides): ghosts against the oracle's rows, gradients against its
    explicit transpose."""
    from gpu_util import compare, to_device_innermost
    w = synth.cubed_sphere(12, 3, 6, 5, ("h", "u", "v"), dtype, seed=21)
    for a in w["fields"]:
        a[np.isnan(a)] = 0.0
    ts = (to_device_innermost if layout == "level_innermost" else to_device)(w["fields"])
    cot = synth.cotangent_like(w, 22)
    _, fwd, grads = _autograd(w, ts, cot)
    op = build_operator(w)
    compare(w, fwd, op=op)
    _check_adjoint(w, cot, grads, op=op)


@pytest.mark.parametrize("layout", ["level_outermost", "level_innermost"])
def test_autograd_full_768_sampled(layout):
    """The differentiation workload at its own size: 6 x 768^2 panels,
    h = 3, (h, u, v) x 32 levels FP32, 6-point interpolation with rotation,
    through BCFill forward and backward in both level layouts; levels 2 and
    29 against the oracle (forward rows and explicit transpose)."""
    from gpu_util import compare, to_device_innermost
    w = synth.adjoint_cubed_sphere()
    ts = (to_device_innermost if layout == "level_innermost" else to_device)(w["fields"])
    cot = synth.cotangent_like(w, 5)
    _, fwd, grads = _autograd(w, ts, cot)
    del ts
    op = build_operator(w, levels=[2, 29])
    compare(w, fwd, op=op, levels=[2, 29])
    _check_adjoint(w, cot, grads, levels=[2, 29], op=op)


def test_mismatched_layout_raises():
    """A plan built for one layout refuses tensors with other strides, a
    wrong dtype or a wrong shape, in the tensor API and in BCFill."""
    import torch
    from gpu_util import to_device_innermost
    w = synth.cubed_sphere(8, 2, 4, 3, ("h", "u", "v"), "f32", seed=23)
    outer = to_device(w["fields"])
    inner = to_device_innermost(w["fields"])
    plan = bc.plan_for_workload(w, outer)
    with pytest.raises(ValueError, match="stride"):
        plan.apply_(inner)
    with pytest.raises(ValueError, match="stride"):
        plan.adjoint_(inner)
    with pytest.raises(ValueError, match="stride"):
        bc.BCFill.apply(plan, *inner)
    with pytest.raises(ValueError, match="dtype"):
        plan.apply_([t.double() for t in outer])
    with pytest.raises(ValueError, match="blocks"):
        plan.apply_(outer[:-1])
    plan.apply_(outer)
    torch.cuda.synchronize()
