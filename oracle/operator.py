"""Explicit assembly and application of ``F(x) = A x + b`` (Sec. III-B).

TEST INFRASTRUCTURE ONLY (see the package docstring).

``A`` has one row per full-region value and one column per data value
(``A_(|R_F|, |R_D|)``); only ghost rows covered by some basic sub-matrix are
populated, and every column must be a data value (columns in the data region
only, so one pass suffices).  Two sub-matrices covering the same ghost value
are rejected.  The in-place apply overwrites covered ghosts with
``A x_D + b`` in FP64, each row summed sequentially in ascending column
order; the adjoint of that in-place map is ``x_D_bar = y_D_bar + A^T y_G_bar``
and ``x_G_bar = 0`` on covered ghosts (their input is overwritten).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .regions import Layout
from .rows import (OracleError, concat_rowsets, const_rows, csr_rows,
                   faces_rows, interp_rows, map_rows, sync_rows, zero_rows)
from .sphere import cubed_sphere_rows

__all__ = ["OracleError", "Operator", "rowsets", "build_operator", "apply",
           "apply_adjoint", "row_scale"]


def rowsets(w, diagnostics=None):
    """Row sets of every boundary description of workload ``w``."""
    blocks = w["blocks"]
    out = []
    for bc in w["bcs"]:
        k = bc["kind"]
        if k == "zero":
            out.append(zero_rows(bc))
        elif k == "const":
            out.append(const_rows(bc))
        elif k == "map":
            out.append(map_rows(bc))
        elif k == "csr":
            out.append(csr_rows(bc))
        elif k == "interp":
            out.append(interp_rows(bc))
        elif k == "faces":
            out.append(faces_rows(bc, blocks))
        elif k == "cubed_sphere_edges":
            out.extend(cubed_sphere_rows(bc, blocks, diagnostics))
        elif k == "sync":
            out.append(sync_rows(bc))
        else:
            raise OracleError(f"unknown boundary kind {k}")
    return [r for r in out if r is not None]


class Operator:
    """``A`` restricted to its covered rows: ``rows`` (sorted row ids),
    ``A`` (CSR, len(rows) x n_data) and ``b`` (len(rows))."""

    def __init__(self, layout, rows, A, b):
        self.layout = layout
        self.rows = rows
        self.A = A
        self.b = b


def _validate(layout, rs, ghost_columns=False):
    b = rs["b"]
    nr = len(rs["c"])
    bb = np.full(nr, b)
    if rs.get("data_rows"):
        # Sync rows (Sec. III-B, block-edge averaging) overwrite data cells
        if not np.all(layout.in_data(bb, rs["ijk"])):
            raise OracleError("a Sync row is not a data cell of its block")
        if np.any(rs["rhs"] != 0.0):
            raise OracleError("a Sync row has b_i != 0")
    elif np.any(layout.in_data(bb, rs["ijk"])) or not np.all(layout.in_full(bb, rs["ijk"])):
        raise OracleError("a row is not a ghost cell of its block")
    if np.any((rs["c"] < 0) | (rs["c"] >= layout.C[b])):
        raise OracleError("row component out of range")
    if len(rs["e_b"]):
        if np.any((rs["e_b"] < 0) | (rs["e_b"] >= layout.nb)):
            raise OracleError("column block out of range")
        inside = layout.in_data(rs["e_b"], rs["e_ijk"])
        if ghost_columns and not rs.get("data_rows"):
            inside = layout.in_full(rs["e_b"], rs["e_ijk"])
        if not np.all(inside):
            raise OracleError("a column is not a data cell")
        if np.any((rs["e_c"] < 0) | (rs["e_c"] >= layout.C[rs["e_b"]])):
            raise OracleError("column component out of range")
        if np.any(layout.L[rs["e_b"]] != layout.L[b]):
            raise OracleError("column block has another level count")
    if not np.all(np.isfinite(rs["e_w"])) or not np.all(np.isfinite(rs["rhs"])):
        raise OracleError("non-finite matrix entry")


def build_operator(w, levels=None, diagnostics=None):
    """Assemble ``A`` and ``b`` of workload ``w``.

    ``levels`` restricts the rows to those levels (for sampled checks of
    large workloads); the columns always span the whole data region.

    With ``w["ghost_sweeps"] = k > 0`` user CSR rows may also read covered
    ghost values (the iterative form HOPE(I) of Sec. II-B): every ghost
    starts at zero and all covered rows are evaluated together ``k`` times
    (Jacobi sweeps), which is the single matrix of HOPE(M),
    ``A = sum_{m<k} G^m D``, ``b = sum_{m<k} G^m b_0`` with ``D`` the entries
    on data values and ``G`` those on ghost values.
    """
    layout = Layout(w["blocks"])
    sets = rowsets(w, diagnostics)
    sweeps = int(w.get("ghost_sweeps") or 0)
    # merge per block, check disjointness at one level
    per_block = {}
    for rs in sets:
        _validate(layout, rs, ghost_columns=sweeps > 0)
        per_block.setdefault(rs["b"], []).append(rs)
    for b, lst in per_block.items():
        rs = concat_rowsets(lst) if len(lst) > 1 else lst[0]
        per_block[b] = rs
        key = layout.row(np.full(len(rs["c"]), b), rs["c"], 0, rs["ijk"])
        if len(np.unique(key)) != len(key):
            raise OracleError("two sub-matrices cover the same value")
    R, Cc, V, Bv, Er = [], [], [], [], []
    row_off = 0
    for b, rs in sorted(per_block.items()):
        nr = len(rs["c"])
        lv = range(int(layout.L[b])) if levels is None else \
            [lv for lv in levels if lv < layout.L[b]]
        for lev in lv:
            R.append(layout.row(np.full(nr, b), rs["c"], lev, rs["ijk"]))
            Bv.append(rs["rhs"])
            if len(rs["e_row"]):
                ghost = ~layout.in_data(rs["e_b"], rs["e_ijk"])
                # data values by column id; ghost values (sweeps only) by
                # -1 - their full-region id, resolved below
                col = np.where(ghost, 0, layout.col(rs["e_b"], rs["e_c"], lev,
                                                    np.where(ghost[:, None], 0, rs["e_ijk"])))
                col = np.where(ghost, -1 - layout.row(rs["e_b"], rs["e_c"], lev, rs["e_ijk"]),
                               col)
                Cc.append(col)
                V.append(rs["e_w"])
                Er.append(rs["e_row"] + row_off)
            row_off += nr
    if not R:
        return Operator(layout, np.zeros(0, np.int64),
                        sp.csr_matrix((0, layout.n_data)), np.zeros(0))
    rows = np.concatenate(R)
    bvec = np.concatenate(Bv)
    order = np.argsort(rows, kind="stable")
    inv = np.empty_like(order)
    inv[order] = np.arange(len(order))
    rows = rows[order]
    bvec = bvec[order]
    if Cc:
        er = inv[np.concatenate(Er)]
        cc = np.concatenate(Cc)
        vv = np.concatenate(V)
        d = cc >= 0
        A = sp.csr_matrix((vv[d], (er[d], cc[d])), shape=(len(rows), layout.n_data))
        if not np.all(d):
            gid = -1 - cc[~d]
            pos = np.searchsorted(rows, gid)
            pos = np.minimum(pos, len(rows) - 1)
            if not np.all(rows[pos] == gid):
                raise OracleError("a column is a ghost value no sub-matrix covers")
            G = sp.csr_matrix((vv[~d], (er[~d], pos)), shape=(len(rows), len(rows)))
            A, bvec = _jacobi_sweeps(A, G, bvec, sweeps)
    else:
        A = sp.csr_matrix((len(rows), layout.n_data))
    A.sum_duplicates()
    A.sort_indices()
    return Operator(layout, rows, A, bvec)


def _jacobi_sweeps(D, G, b0, k):
    """``k`` Jacobi sweeps from zero ghosts, ``g <- D x + G g + b0``, as one
    affine map of the data: ``(A, b)`` with ``A_0 = 0, b_0 = 0``,
    ``A_{m+1} = D + G A_m``, ``b_{m+1} = b0 + G b_m``."""
    A = sp.csr_matrix(D.shape)
    b = np.zeros(len(b0))
    for _ in range(k):
        A = (D + G @ A).tocsr()
        b = b0 + G @ b
    return A, b


def apply(op, fields):
    """In-place ghost fill: returns FP64 copies of ``fields`` with every
    covered ghost replaced by ``(A x_D + b)_i``."""
    lay = op.layout
    y = lay.flatten_full(fields)
    x = lay.data_vector(fields)
    y[op.rows] = op.A @ x + op.b
    return lay.unflatten_full(y, fields)


def ghost_values(op, fields):
    """``A x_D + b`` on the covered rows only (row order of ``op.rows``)."""
    return op.A @ op.layout.data_vector(fields) + op.b


def row_scale(op, fields):
    """``sum_e |A_ie| |x_e| + |b_i|`` per covered row: the scale of the
    rounding error of any evaluation order of row ``i``."""
    x = np.abs(op.layout.data_vector(fields))
    return abs(op.A) @ x + np.abs(op.b)


def apply_adjoint(op, cot):
    """Adjoint of the in-place fill ``out_i = (A x_D + b)_i`` on the covered
    rows, ``out_j = x_j`` elsewhere, applied to cotangent ``cot``:
    ``x_bar_j = [j not covered] y_bar_j + sum_i A_ij y_bar_i``.  Covered rows
    are ghosts (whose x_bar is 0) and, with block-edge averaging, data cells
    (whose own y_bar is consumed by their row); uncovered values pass through.
    """
    lay = op.layout
    y = lay.flatten_full(cot)
    g = y[op.rows].copy()
    contrib = op.A.T @ g
    y[op.rows] = 0.0
    y[lay.data_rows()] += contrib
    return lay.unflatten_full(y, cot)
