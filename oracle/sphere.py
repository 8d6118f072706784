"""Cubed-sphere panel-edge interpolation rows (Sec. III-B, user-defined
interpolation ``A_ij = Itp_ij``; Sec. V-A, vector components).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper leaves the geometry to the user; this oracle fixes the reading used
throughout the project:

* Panels are equiangular gnomonic.  A panel ``P`` has an outward normal
  ``n_P`` and two in-face unit axes ``ex_P``, ``ey_P``; the cube point of
  angles ``(a, b)`` is ``n_P + tan(a) ex_P + tan(b) ey_P`` and its projection
  onto the unit sphere is the grid point.  Panels 0..3 face +X, +Y, -X, -Y,
  panel 4 faces +Z and panel 5 faces -Z.
* Cell ``i`` of an ``N``-cell axis has angle ``-pi/4 + (i + 1/2) pi/(2N)``,
  ghost cells included.
* An edge ghost (one index out of range) is mapped to the panel ``Q`` whose
  normal has the largest projection on it.  One fractional index of that
  point on ``Q`` is a data row ``r'`` (exactly, up to rounding); the other is
  the along-edge position ``t``.
* If ``t`` is within 1e-9 of an integer inside ``[0, N)`` the row is a unit
  copy ("copies where grid lines align").  Otherwise it interpolates along
  row ``r'`` with the ``p`` nodes ``start .. start + p - 1``,
  ``start = clamp(floor(t) - (p/2 - 1), 0, N - p)``, by the Lagrange basis
  ``w_k = prod_{m != k} (tau - m) / (k - m)`` at ``tau = t - start``.
* Vector components are covariant, ``u_i = V . dr/d(a_i)`` on the unit
  sphere.  The ghost value is ``u_own = M u_nb`` with ``u_nb`` the
  interpolated components of ``Q`` and ``M_ij = e_own_i . e_Q^j``, ``e^j``
  being ``Q``'s dual basis at the ghost point (interpolate, then rotate).
* Reconstruction-and-quadrature rows (``quad = nq``, the finite-volume form
  of Sec. II-B written as ``Itp = Agg . Recons``, Sec. III-B): data values
  are cell averages in the panel's angle coordinates.  An edge ghost cell is
  the average of ``nq x nq`` Gauss-Legendre points of the cell in its own
  panel's angles (weights ``w_a w_b / 4``); each point is carried to ``Q``
  and evaluated there by the tensor-product polynomial of degree ``p - 1``
  per axis whose averages over a ``p x p`` patch of ``Q``'s data cells are
  the data values.  The patch is chosen once per ghost from its centre:
  normal cells from ``clamp(r' - (p/2 - 1), 0, N - p)``, along cells from
  ``clamp(floor(t + 1e-9) - (p/2 - 1), 0, N - p)``.  Vector pairs are
  rotated by ``M`` at every point before the average.  With ``centred`` the
  two clamps are dropped: near the panel corners and across the shared
  edge the patch then takes ghost cells of ``Q`` (HOPE(I) of Sec. II-B),
  which the operator resolves by Jacobi sweeps (``ghost_sweeps``).
"""
from __future__ import annotations

import math

import numpy as np

from .rows import OracleError, concat_rowsets, empty_rowset

# outward normal, x axis and y axis of each panel
PANEL_FRAME = np.array([
    [[1, 0, 0], [0, 1, 0], [0, 0, 1]],
    [[0, 1, 0], [-1, 0, 0], [0, 0, 1]],
    [[-1, 0, 0], [0, -1, 0], [0, 0, 1]],
    [[0, -1, 0], [1, 0, 0], [0, 0, 1]],
    [[0, 0, 1], [0, 1, 0], [-1, 0, 0]],
    [[0, 0, -1], [0, 1, 0], [1, 0, 0]],
], dtype=np.float64)

SNAP_TOL = 1e-9


def angle(N, i):
    return -math.pi / 4 + (np.asarray(i, np.float64) + 0.5) * (math.pi / (2 * N))


def sphere_point(P, a, b):
    """Unit vector of panel ``P`` at angles (a, b)."""
    nrm, ex, ey = PANEL_FRAME[P]
    a, b = np.broadcast_arrays(np.asarray(a, np.float64), np.asarray(b, np.float64))
    F = (nrm[None, :] + np.tan(a).reshape(-1, 1) * ex[None, :]
         + np.tan(b).reshape(-1, 1) * ey[None, :])
    return F / np.linalg.norm(F, axis=1, keepdims=True)


def locate(v):
    """Panel containing unit vectors ``v`` (largest normal projection) and
    the angles there."""
    v = np.asarray(v, np.float64).reshape(-1, 3)
    proj = v @ PANEL_FRAME[:, 0, :].T            # (n, 6)
    Q = np.argmax(proj, axis=1)
    nrm = PANEL_FRAME[Q, 0, :]
    ex = PANEL_FRAME[Q, 1, :]
    ey = PANEL_FRAME[Q, 2, :]
    dn = np.sum(v * nrm, axis=1)
    a = np.arctan(np.sum(v * ex, axis=1) / dn)
    b = np.arctan(np.sum(v * ey, axis=1) / dn)
    return Q, a, b


def covariant_basis(P, a, b):
    """``dr/da`` and ``dr/db`` of the unit position on panel ``P``."""
    nrm, ex, ey = PANEL_FRAME[P]
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    F = nrm[None, :] + np.tan(a)[:, None] * ex[None, :] + np.tan(b)[:, None] * ey[None, :]
    nF = np.linalg.norm(F, axis=1, keepdims=True)
    r = F / nF
    sa = 1.0 / np.cos(a) ** 2
    sb = 1.0 / np.cos(b) ** 2
    ea = sa[:, None] * (ex[None, :] - r * (r @ ex)[:, None]) / nF
    eb = sb[:, None] * (ey[None, :] - r * (r @ ey)[:, None]) / nF
    return ea, eb


def dual_basis(ea, eb):
    g11 = np.sum(ea * ea, axis=1)
    g12 = np.sum(ea * eb, axis=1)
    g22 = np.sum(eb * eb, axis=1)
    det = g11 * g22 - g12 * g12
    da = (g22[:, None] * ea - g12[:, None] * eb) / det[:, None]
    db = (-g12[:, None] * ea + g11[:, None] * eb) / det[:, None]
    return da, db


def lagrange_weights(tau, p):
    """Lagrange basis of the nodes 0..p-1 evaluated at ``tau`` (n, p)."""
    tau = np.asarray(tau, np.float64).reshape(-1)
    w = np.ones((len(tau), p), np.float64)
    for k in range(p):
        for m in range(p):
            if m != k:
                w[:, k] *= (tau - m) / (k - m)
    return w


def edge_strip_cells(N, h, d, side):
    """Ghost cells of the edge strip beyond axis ``d``'s ``side``: depth
    ``r`` (0 next to the data) and along index ``s``; cells (n, 3)."""
    r = np.repeat(np.arange(h), N)
    s = np.tile(np.arange(N), h)
    cells = np.zeros((h * N, 3), np.int64)
    cells[:, d] = (-1 - r) if side == 0 else (N + r)
    cells[:, 1 - d] = s
    return cells, r, s


def strip_geometry(P, N, h, d, side):
    """Neighbour panel and per-cell stencil data of one edge strip.

    Returns a dict with ``Q``, ``dq`` (the axis of Q normal to the shared
    edge), per-cell ``cells``, ``rq`` (depth row on Q), ``t`` (along
    position on Q), ``a``, ``b`` (ghost angles on P) and ``aq``, ``bq``
    (the same point's angles on Q)."""
    delta = math.pi / (2 * N)
    depth_ang = (math.pi / 4 + delta / 2) * (1 if side == 1 else -1)
    ref = [0.0, 0.0]
    ref[d] = depth_ang
    Qr, ar, br = locate(sphere_point(P, ref[0], ref[1]))
    Q = int(Qr[0])
    dq = 0 if abs(ar[0]) > abs(br[0]) else 1
    q_side = 1 if (ar[0] if dq == 0 else br[0]) > 0 else 0

    cells, r, s = edge_strip_cells(N, h, d, side)
    a = angle(N, cells[:, 0])
    b = angle(N, cells[:, 1])
    Qc, aq, bq = locate(sphere_point(P, a, b))
    if np.any(Qc != Q):
        raise OracleError("edge strip spans more than one neighbour panel")
    fq = [(aq + math.pi / 4) / delta - 0.5, (bq + math.pi / 4) / delta - 0.5]
    fdepth, t = fq[dq], fq[1 - dq]
    rq = np.rint(fdepth).astype(np.int64)
    if np.any(np.abs(fdepth - rq) > SNAP_TOL):
        raise OracleError("ghost point is not on a data row of the neighbour")
    expect = r if q_side == 0 else N - 1 - r
    if np.any(rq != expect):
        raise OracleError("neighbour depth row does not match the ghost depth")
    return {"Q": Q, "dq": dq, "q_side": q_side, "cells": cells, "r": r,
            "s": s, "rq": rq, "t": t, "a": a, "b": b, "aq": aq, "bq": bq}


def stencil(t, N, p):
    """Snap flags, stencil start and weights of along positions ``t``."""
    tr = np.rint(t)
    snapped = (np.abs(t - tr) < SNAP_TOL) & (tr >= 0) & (tr <= N - 1)
    start = np.clip(np.floor(t).astype(np.int64) - (p // 2 - 1), 0, N - p)
    w = lagrange_weights(t - start, p)
    start = np.where(snapped, tr.astype(np.int64), start)
    return snapped, start, w


def rotation(P, Q, a, b, aq, bq):
    """``M`` (n, 2, 2) with ``M_ij = e_P_i . e_Q^j`` at the ghost points."""
    ea, eb = covariant_basis(P, a, b)
    qa, qb = covariant_basis(Q, aq, bq)
    da, db = dual_basis(qa, qb)
    M = np.empty((len(ea), 2, 2))
    for i, e in enumerate((ea, eb)):
        for j, dd in enumerate((da, db)):
            M[:, i, j] = np.sum(e * dd, axis=1)
    return M


def cubed_sphere_rows(bc, blocks, diagnostics=None):
    """Row sets (one per panel) of the panel-edge interpolation; with a
    ``quad`` entry, the reconstruction-and-quadrature rows of
    :func:`cubed_sphere_quad_rows`."""
    if bc.get("quad"):
        return cubed_sphere_quad_rows(bc, blocks)
    panels = list(bc["panels"])
    N, h, p = int(bc["N"]), int(bc["h"]), int(bc["p"])
    if p > N:
        raise OracleError("stencil wider than the panel")
    scal = list(bc["scalar_comps"])
    vpair = bc.get("vector_pair")
    for pb in panels:
        blk = blocks[pb]
        if tuple(blk["n"][:2]) != (N, N) or tuple(blk["h"][:2]) != (h, h):
            raise OracleError("panel block shape does not match N, h")
    out = []
    for P in range(6):
        sets = []
        for d in (0, 1):
            for side in (0, 1):
                g = strip_geometry(P, N, h, d, side)
                snapped, start, w = stencil(g["t"], N, p)
                R = len(g["cells"])
                # source cells of every stencil node
                nodes_k = np.where(snapped[:, None], 0,
                                   np.arange(p)[None, :])      # (R, p)
                src = np.zeros((R, p, 3), np.int64)
                src[:, :, g["dq"]] = g["rq"][:, None]
                src[:, :, 1 - g["dq"]] = start[:, None] + nodes_k
                wk = np.where(snapped[:, None],
                              (np.arange(p) == 0)[None, :].astype(np.float64), w)
                keep = np.broadcast_to(~snapped[:, None] | (np.arange(p) == 0)[None, :],
                                       (R, p))
                e_row = np.broadcast_to(np.arange(R)[:, None], (R, p))[keep]
                e_src = src[keep]
                e_w = wk[keep]
                Qb = panels[g["Q"]]
                for c in scal:
                    rs = empty_rowset(panels[P], np.full(R, c), g["cells"])
                    rs["e_row"] = e_row.copy()
                    rs["e_b"] = np.full(len(e_row), Qb, np.int64)
                    rs["e_c"] = np.full(len(e_row), c, np.int64)
                    rs["e_ijk"] = e_src.copy()
                    rs["e_w"] = e_w.copy()
                    sets.append(rs)
                if vpair:
                    M = rotation(P, g["Q"], g["a"], g["b"], g["aq"], g["bq"])
                    cu, cv = vpair
                    for i, c_row in enumerate((cu, cv)):
                        rs = empty_rowset(panels[P], np.full(R, c_row), g["cells"])
                        rows, bb, cc, ijk, ww = [], [], [], [], []
                        for j, c_col in enumerate((cu, cv)):
                            rows.append(e_row)
                            bb.append(np.full(len(e_row), Qb, np.int64))
                            cc.append(np.full(len(e_row), c_col, np.int64))
                            ijk.append(e_src)
                            ww.append(M[e_row, i, j] * e_w)
                        rs["e_row"] = np.concatenate(rows)
                        rs["e_b"] = np.concatenate(bb)
                        rs["e_c"] = np.concatenate(cc)
                        rs["e_ijk"] = np.concatenate(ijk)
                        rs["e_w"] = np.concatenate(ww)
                        sets.append(rs)
                if diagnostics is not None:
                    diagnostics.append({"P": P, "d": d, "side": side, "Q": g["Q"],
                                        "dq": g["dq"], "q_side": g["q_side"],
                                        "cells": g["cells"], "r": g["r"],
                                        "s": g["s"], "rq": g["rq"], "t": g["t"],
                                        "snapped": snapped, "start": start,
                                        "w": w})
        out.append(concat_rowsets(sets))
    return out


# ----------------------------------------------------------------------------
# Reconstruction at quadrature points (Sec. II-B, the HOPE example; Sec. III-B,
# Itp = Agg . Recons)
# ----------------------------------------------------------------------------
def patch_starts(rq, t, N, p, centred=False):
    """First node of the ``p x p`` reconstruction patch on the neighbour panel
    along its normal axis (from the depth row ``rq``) and along the edge (from
    the along position ``t`` of the ghost centre).  Clamped into the data
    cells, or, ``centred``, left centred on the ghost (the patch may then
    take ghost cells of the neighbour, the HOPE(I) case of Sec. II-B)."""
    sn = np.asarray(rq, np.int64) - (p // 2 - 1)
    st = np.floor(np.asarray(t) + SNAP_TOL).astype(np.int64) - (p // 2 - 1)
    if not centred:
        sn, st = np.clip(sn, 0, N - p), np.clip(st, 0, N - p)
    return sn, st


def average_reconstruction_weights(x, p):
    """Weights ``c_k(x)`` (n, p) of the polynomial of degree ``p - 1`` whose
    averages over the unit cells ``[k - 1/2, k + 1/2]``, ``k = 0..p-1``, are
    given: ``P(x) = sum_k c_k(x) avg_k``.

    Written from the primitive ``Phi(x) = int_{-1/2}^x P``: ``Phi`` is known
    at the cell edges ``e_m = m - 1/2`` (``Phi(e_m) = sum_{k<m} avg_k``), is
    the degree-``p`` Lagrange interpolant ``sum_m Phi(e_m) l_m(x)`` through
    them, and ``P = Phi'``, so ``c_k = sum_{m > k} l_m'``."""
    x = np.asarray(x, np.float64).reshape(-1)
    e = np.arange(p + 1, dtype=np.float64) - 0.5
    dl = np.zeros((len(x), p + 1))
    for m in range(p + 1):
        for j in range(p + 1):
            if j == m:
                continue
            term = np.full(len(x), 1.0 / (e[m] - e[j]))
            for i in range(p + 1):
                if i != m and i != j:
                    term *= (x - e[i]) / (e[m] - e[i])
            dl[:, m] += term
    c = np.zeros((len(x), p))
    for k in range(p):
        for m in range(k + 1, p + 1):
            c[:, k] += dl[:, m]
    return c


def quad_strip(P, N, h, p, nq, d, side, vector, centred=False):
    """Weights of the ghost cells of one edge strip.

    Each ghost cell is averaged over its ``nq x nq`` Gauss-Legendre points in
    the panel's own angles (``Agg``: weights ``w_a w_b / 4``); each point is
    carried to the neighbour panel ``Q`` and reconstructed there from the
    cell averages of the ``p x p`` data cells of the ghost's patch, one
    :func:`average_reconstruction_weights` factor per axis (``Recons``).  Returns the strip geometry, the patch
    starts and ``W[R, p, p]`` (scalar rows, normal node first) and, for a
    vector pair, ``V[R, 2, 2, p, p]`` with ``V[:, i, j]`` the weights of
    neighbour component ``j`` in own component ``i`` (rotation applied at
    every point)."""
    g = strip_geometry(P, N, h, d, side)
    Q, dq = g["Q"], g["dq"]
    sn, st = patch_starts(g["rq"], g["t"], N, p, centred)
    if np.any(sn < -h) or np.any(sn + p > N + h) or np.any(st < -h) or np.any(st + p > N + h):
        raise OracleError("a centred patch leaves the neighbour's full region")
    xg, wg = np.polynomial.legendre.leggauss(nq)
    delta = math.pi / (2 * N)
    R = len(g["cells"])
    W = np.zeros((R, p, p))
    V = np.zeros((R, 2, 2, p, p)) if vector else None
    for ia in range(nq):
        for ib in range(nq):
            a = g["a"] + xg[ia] * delta / 2
            b = g["b"] + xg[ib] * delta / 2
            Qc, aq, bq = locate(sphere_point(P, a, b))
            if np.any(Qc != Q):
                raise OracleError("a quadrature point leaves the neighbour panel")
            f = [(aq + math.pi / 4) / delta - 0.5, (bq + math.pi / 4) / delta - 0.5]
            Ln = average_reconstruction_weights(f[dq] - sn, p)
            Lt = average_reconstruction_weights(f[1 - dq] - st, p)
            omega = wg[ia] * wg[ib] / 4.0
            T = omega * Ln[:, :, None] * Lt[:, None, :]
            W += T
            if vector:
                M = rotation(P, Q, a, b, aq, bq)
                for i in range(2):
                    for j in range(2):
                        V[:, i, j] += M[:, i, j, None, None] * T
    return g, sn, st, W, V


def cubed_sphere_quad_rows(bc, blocks):
    """Row sets (one per panel) of the reconstruction-and-quadrature rows:
    every edge ghost reads the ``p x p`` patch of neighbour data cells
    (entries normal node major, along node minor)."""
    panels = list(bc["panels"])
    N, h, p, nq = int(bc["N"]), int(bc["h"]), int(bc["p"]), int(bc["quad"])
    centred = bool(bc.get("centred"))
    if p < 2 or p > N:
        raise OracleError("reconstruction order must be in 2..N")
    if nq < 1:
        raise OracleError("at least one quadrature point per axis")
    scal = list(bc["scalar_comps"])
    vpair = bc.get("vector_pair")
    for pb in panels:
        blk = blocks[pb]
        if tuple(blk["n"][:2]) != (N, N) or tuple(blk["h"][:2]) != (h, h):
            raise OracleError("panel block shape does not match N, h")
    kn, kt = np.meshgrid(np.arange(p), np.arange(p), indexing="ij")
    kn, kt = kn.reshape(-1), kt.reshape(-1)
    out = []
    for P in range(6):
        sets = []
        for d in (0, 1):
            for side in (0, 1):
                g, sn, st, W, V = quad_strip(P, N, h, p, nq, d, side, bool(vpair), centred)
                R = len(g["cells"])
                src = np.zeros((R, p * p, 3), np.int64)
                src[:, :, g["dq"]] = sn[:, None] + kn[None, :]
                src[:, :, 1 - g["dq"]] = st[:, None] + kt[None, :]
                e_row = np.repeat(np.arange(R), p * p)
                e_src = src.reshape(-1, 3)
                Qb = panels[g["Q"]]
                for c in scal:
                    rs = empty_rowset(panels[P], np.full(R, c), g["cells"])
                    rs["e_row"] = e_row.copy()
                    rs["e_b"] = np.full(len(e_row), Qb, np.int64)
                    rs["e_c"] = np.full(len(e_row), c, np.int64)
                    rs["e_ijk"] = e_src.copy()
                    rs["e_w"] = W.reshape(-1).copy()
                    sets.append(rs)
                if vpair:
                    cu, cv = vpair
                    for i, c_row in enumerate((cu, cv)):
                        rs = empty_rowset(panels[P], np.full(R, c_row), g["cells"])
                        rs["e_row"] = np.concatenate([e_row, e_row])
                        rs["e_b"] = np.full(2 * len(e_row), Qb, np.int64)
                        rs["e_c"] = np.concatenate([np.full(len(e_row), cu, np.int64),
                                                    np.full(len(e_row), cv, np.int64)])
                        rs["e_ijk"] = np.concatenate([e_src, e_src])
                        rs["e_w"] = np.concatenate([V[:, i, 0].reshape(-1),
                                                    V[:, i, 1].reshape(-1)])
                        sets.append(rs)
        out.append(concat_rowsets(sets))
    return out
