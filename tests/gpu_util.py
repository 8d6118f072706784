"""Helpers of the GPU parity tests: run a workload through the C ABI and
compare it with the FP64 oracle (bit-exact on copy / zero / constant rows,
row-scaled tolerance on interpolation and CSR rows)."""
import numpy as np

from oracle.operator import build_operator, row_scale
from paper_2605_14780_gb300 import bc

TOL = {"f64": 1e-12, "f32": 2e-6}


def to_device(fields):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields]


def to_device_innermost(fields):
    """Device copies with every component stored [k][j][i][level]; the views
    keep the (C, L, F2, F1, F0) index order."""
    import torch
    out = []
    for a in fields:
        base = torch.from_numpy(np.ascontiguousarray(a.transpose(0, 2, 3, 4, 1))).cuda()
        out.append(base.permute(0, 4, 1, 2, 3))
    return out


def run(w, form=bc.BC_FORM_BATCHED, opts=None, tensors=None, repeat=1):
    import torch
    ts = tensors if tensors is not None else to_device(w["fields"])
    plan = bc.plan_for_workload(w, ts, opts)
    table = bc.slot_table(ts)
    for _ in range(repeat):
        plan.apply(table, form)
    torch.cuda.synchronize()
    return plan, [t.cpu().numpy() for t in ts]


def flat(arrs):
    return np.concatenate([np.asarray(a).ravel() for a in arrs])


def bits(a):
    a = np.asarray(a)
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


def compare(w, out, op=None, levels=None):
    """Check GPU output ``out`` (list of arrays) against the oracle."""
    op = op or build_operator(w, levels=levels)
    dt = np.float32 if w["dtype"] == "f32" else np.float64
    tol = TOL[w["dtype"]]
    x = op.layout.data_vector(w["fields"])
    g = op.A @ x + op.b
    scale = row_scale(op, w["fields"])
    got_all = flat(out)
    src_all = flat(w["fields"])
    got = got_all[op.rows].astype(np.float64)
    nnz = np.diff(op.A.indptr)
    unit = (nnz == 1) & (op.b == 0)
    unit[unit] = op.A.data[op.A.indptr[:-1][unit]] == 1.0
    exact = (nnz == 0) | unit
    # bit-exact rows: oracle value rounded to the dtype
    ge = bits(got_all[op.rows][exact])
    oe = bits(g[exact].astype(dt))
    bad = np.nonzero(ge != oe)[0]
    assert len(bad) == 0, f"{len(bad)} copy/zero rows differ, e.g. row {op.rows[exact][bad[0]]}"
    # tolerance rows
    err = np.abs(got[~exact] - g[~exact])
    lim = tol * scale[~exact]
    worst = np.max(err / np.maximum(lim, 1e-300)) if err.size else 0.0
    assert np.all(err <= lim), f"row-scaled error {worst} x tol"
    if err.size:
        gmax = np.max(np.abs(g[~exact]))
        assert np.max(err) <= tol * max(gmax, 1e-300) * 10
    # every value that is not a covered ghost is untouched (full restriction
    # only: with sampled levels the other levels are covered as well)
    if levels is None:
        mask = np.ones(got_all.size, bool)
        mask[op.rows] = False
        assert np.array_equal(bits(got_all[mask]), bits(src_all[mask]))
    return op, int(exact.sum()), int((~exact).sum())
