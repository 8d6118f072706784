"""Sparse rows of the structured and user-CSR boundary conditions (Sec. III-B).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Each function returns a *row set*: the rows one basic sub-matrix contributes at
a single level, as plain arrays

    b      int            destination block
    c      int[R]         component of each row
    ijk    int[R, 3]      ghost cell of each row
    e_row  int[E]         row (0..R-1) of each entry
    e_b, e_c, e_ijk       block, component and data cell of each entry column
    e_w    float64[E]     entry value A_ij
    rhs    float64[R]     b_i

A row set is repeated at every level of its block, reading the same level of
its column blocks.
"""
from __future__ import annotations

import numpy as np

from .regions import box_cells, ghost_cells


class OracleError(ValueError):
    """An invalid operator description (overlap, non-data column, ...)."""


def empty_rowset(b, c, ijk):
    R = len(ijk)
    return {"b": int(b), "c": np.asarray(c, np.int64).reshape(R),
            "ijk": np.asarray(ijk, np.int64).reshape(R, 3),
            "e_row": np.zeros(0, np.int64), "e_b": np.zeros(0, np.int64),
            "e_c": np.zeros(0, np.int64), "e_ijk": np.zeros((0, 3), np.int64),
            "e_w": np.zeros(0, np.float64), "rhs": np.zeros(R, np.float64)}


def unit_rowset(b, c, ijk, src_b, src_c, src_ijk):
    """Rows with a single unit entry ``A_ij = 1`` (halo copy, circular and
    symmetric maps; Sec. III-B)."""
    rs = empty_rowset(b, c, ijk)
    R = len(rs["c"])
    rs["e_row"] = np.arange(R, dtype=np.int64)
    rs["e_b"] = np.broadcast_to(np.asarray(src_b, np.int64), (R,)).copy()
    rs["e_c"] = np.broadcast_to(np.asarray(src_c, np.int64), (R,)).copy()
    rs["e_ijk"] = np.asarray(src_ijk, np.int64).reshape(R, 3)
    rs["e_w"] = np.ones(R, np.float64)
    return rs


def concat_rowsets(sets):
    """Merge row sets of the same block into one."""
    sets = [s for s in sets if len(s["c"])]
    if not sets:
        return None
    b = sets[0]["b"]
    out = empty_rowset(b, np.concatenate([s["c"] for s in sets]),
                       np.concatenate([s["ijk"] for s in sets]))
    off, er = 0, []
    for s in sets:
        assert s["b"] == b
        er.append(s["e_row"] + off)
        off += len(s["c"])
    out["e_row"] = np.concatenate(er)
    for key in ("e_b", "e_c", "e_w"):
        out[key] = np.concatenate([s[key] for s in sets])
    out["e_ijk"] = np.concatenate([s["e_ijk"] for s in sets]).reshape(-1, 3)
    out["rhs"] = np.concatenate([s["rhs"] for s in sets])
    return out


def _comps_cells(comps, cells):
    """Rows ordered component-major, then cell."""
    comps = list(comps)
    c = np.repeat(np.asarray(comps, np.int64), len(cells))
    ijk = np.tile(cells, (len(comps), 1))
    return c, ijk


# ----------------------------------------------------------------------------
# fmap: circular and symmetric boundaries (Sec. III-B)
# ----------------------------------------------------------------------------
def fmap(i, N, kind):
    """Index map of a circular or symmetric boundary along one axis.

    The paper gives the left side: the ghost at coordinate ``-x`` maps to
    ``x - 1`` (symmetric) or ``|R_D| - x`` (circular), ``0 < x``.  The right
    side is its mirror image: the ghost at ``N - 1 + x`` maps to ``N - x``
    (symmetric) or ``x - 1`` (circular).  Coordinates inside ``[0, N)`` are
    returned unchanged.  Every image must land in ``[0, N)``, which bounds the
    ghost depth by ``x <= N``.
    """
    i = np.asarray(i, np.int64)
    out = i.copy()
    left, right = i < 0, i >= N
    xl = -i[left]
    xr = i[right] - (N - 1)
    if np.any(xl > N) or np.any(xr > N):
        raise OracleError("halo deeper than the data region for fmap")
    if kind == "symmetric":
        out[left] = xl - 1
        out[right] = N - xr
    elif kind == "circular":
        out[left] = N - xl
        out[right] = xr - 1
    else:
        raise OracleError(f"unknown fmap kind {kind}")
    return out


# ----------------------------------------------------------------------------
# explicit kinds
# ----------------------------------------------------------------------------
def zero_rows(bc):
    """Zero padding: ``A_ij = b_i = 0`` (Sec. III-B)."""
    c, ijk = _comps_cells(bc["comps"], box_cells(bc["lo"], bc["hi"]))
    return empty_rowset(bc["block"], c, ijk)


def const_rows(bc):
    """Pure-function boundary with the function tabulated: ``A = 0``,
    ``b_i = udf(i)`` (Sec. III-B)."""
    c, ijk = _comps_cells(bc["comps"], box_cells(bc["lo"], bc["hi"]))
    rs = empty_rowset(bc["block"], c, ijk)
    rs["rhs"] = np.asarray(bc["values"], np.float64).reshape(-1).copy()
    if len(rs["rhs"]) != len(c):
        raise OracleError("const values do not match the box")
    return rs


def interp_rows(bc):
    """User-defined interpolation rows ``A_ij = Itp_ij`` (Sec. III-B) given as
    tables: box cell ``q`` reads the ``p`` data cells ``start[q] + n e_axis``
    (``n < p``) of ``src_block`` with weights ``w[q, n]``.  A covariant pair
    ``rot_comp = (cu, cv)`` is interpolated, then multiplied by the 2x2
    ``rot[q]`` (row-major); other listed components use the plain row."""
    cells = box_cells(bc["lo"], bc["hi"])
    R = len(cells)
    p = int(bc["p"])
    start = np.asarray(bc["start"], np.int64).reshape(R, 3)
    axis = np.asarray(bc["axis"], np.int64).reshape(R)
    w = np.asarray(bc["w"], np.float64).reshape(R, p)
    src = np.repeat(start[:, None, :], p, axis=1)               # (R, p, 3)
    src[np.arange(R)[:, None], np.arange(p)[None, :], axis[:, None]] += np.arange(p)[None, :]
    pair = tuple(bc.get("rot_comp") or (-1, -1))
    rot = np.asarray(bc["rot"], np.float64).reshape(R, 2, 2) if pair[0] >= 0 else None
    sets = []
    e_row = np.repeat(np.arange(R), p)
    for c in bc["comps"]:
        rs = empty_rowset(bc["block"], np.full(R, c), cells)
        if c in pair:
            i = pair.index(c)
            rs["e_row"] = np.concatenate([e_row, e_row])
            rs["e_c"] = np.concatenate([np.full(R * p, pair[0]), np.full(R * p, pair[1])])
            rs["e_ijk"] = np.concatenate([src.reshape(-1, 3), src.reshape(-1, 3)])
            rs["e_w"] = np.concatenate([(rot[:, i, 0][:, None] * w).reshape(-1),
                                        (rot[:, i, 1][:, None] * w).reshape(-1)])
        else:
            rs["e_row"] = e_row.copy()
            rs["e_c"] = np.full(R * p, c)
            rs["e_ijk"] = src.reshape(-1, 3).copy()
            rs["e_w"] = w.reshape(-1).copy()
        rs["e_b"] = np.full(len(rs["e_row"]), bc["src_block"], np.int64)
        sets.append(rs)
    return concat_rowsets(sets)


def map_rows(bc):
    """A static single-entry row list (Table III, F_LIST), e.g. the rotated
    map of Alg. 1: the column of ghost ``g`` is
    ``src[d] = sign[d] * g[perm[d]] + offset[d]`` in ``src_block``."""
    cells = box_cells(bc["lo"], bc["hi"])
    perm = np.asarray(bc["perm"], np.int64)
    sign = np.asarray(bc["sign"], np.int64)
    off = np.asarray(bc["offset"], np.int64)
    src = cells[:, perm] * sign[None, :] + off[None, :]
    c, ijk = _comps_cells(bc["comps"], cells)
    src_ijk = np.tile(src, (len(bc["comps"]), 1))
    return unit_rowset(bc["block"], c, ijk, bc["src_block"], c, src_ijk)


def csr_rows(bc):
    """User CSR rows (Table III: F_NNZ, F_COL, F_DATA; the built-in
    BoundaryCSR of Sec. IV-A).  Row ``r`` is ghost cell ``r % volume`` of the
    box for the ``r // volume``-th listed component."""
    cells = box_cells(bc["lo"], bc["hi"])
    c, ijk = _comps_cells(bc["comps"], cells)
    rp = np.asarray(bc["row_ptr"], np.int64)
    if len(rp) != len(c) + 1:
        raise OracleError("row_ptr does not match the box")
    rs = empty_rowset(bc["block"], c, ijk)
    counts = np.diff(rp)
    rs["e_row"] = np.repeat(np.arange(len(c), dtype=np.int64), counts)
    rs["e_b"] = np.asarray(bc["col_block"], np.int64)[rp[0]:rp[-1]]
    rs["e_c"] = np.asarray(bc["col_comp"], np.int64)[rp[0]:rp[-1]]
    rs["e_ijk"] = np.asarray(bc["col_ijk"], np.int64).reshape(-1, 3)[rp[0]:rp[-1]]
    rs["e_w"] = np.asarray(bc["val"], np.float64)[rp[0]:rp[-1]]
    if bc.get("rhs") is not None:
        rs["rhs"] = np.asarray(bc["rhs"], np.float64).copy()
    return rs


def sync_rows(bc):
    """Block-edge averaging (``Sync`` of Sec. III-B): rows on data cells that
    several blocks store for one physical location, ``A_ij = Sync_ij`` over
    the shared data cells, ``b_i = 0``.  Laid out like a CSR sub-matrix whose
    box lies in the data region; the row set is flagged so that validation
    expects data-cell rows."""
    rs = csr_rows(bc)
    rs["data_rows"] = True
    return rs


# ----------------------------------------------------------------------------
# per-face descriptions of one block
# ----------------------------------------------------------------------------
def faces_rows(bc, blocks):
    """Rows of a block whose faces each carry one boundary type.

    A ghost cell with exactly one axis out of range takes its face's rows.
    A ghost cell with several axes out of range (an edge or corner) is zero
    when ``corners == "zero"`` (as the corners of Alg. 1); with
    ``corners == "product"`` it applies every out-of-range axis's circular or
    symmetric map independently, and is zero as soon as one of those faces
    is not a map.
    """
    b = bc["block"]
    blk = blocks[b]
    n = np.asarray(blk["n"], np.int64)
    comps = list(range(blk["ncomp"]))
    face = {(f["axis"], f["side"]): f for f in bc["faces"]}
    G = ghost_cells(blk)
    low = G < 0
    high = G >= n[None, :]
    out = low | high
    nout = out.sum(axis=1)
    sets = []

    def add_zero(cells):
        if len(cells):
            c, ijk = _comps_cells(comps, cells)
            sets.append(empty_rowset(b, c, ijk))

    def add_unit(cells, src_b, src_cells):
        if len(cells):
            c, ijk = _comps_cells(comps, cells)
            sets.append(unit_rowset(b, c, ijk, src_b, c,
                                    np.tile(src_cells, (len(comps), 1))))

    # edges and corners
    multi = nout >= 2
    if np.any(multi):
        cells = G[multi]
        if bc["corners"] == "zero":
            add_zero(cells)
        elif bc["corners"] == "product":
            src = cells.copy()
            is_map = np.ones(len(cells), bool)
            for d in range(3):
                for side, m in ((0, low[multi, d]), (1, high[multi, d])):
                    if not np.any(m):
                        continue
                    f = face.get((d, side))
                    if f is None or f["type"] not in ("circular", "symmetric"):
                        is_map &= ~m
                        continue
                    src[m, d] = fmap(cells[m, d], int(n[d]), f["type"])
            add_zero(cells[~is_map])
            add_unit(cells[is_map], b, src[is_map])
        else:
            raise OracleError(f"unknown corner rule {bc['corners']}")

    # faces
    for (d, side), f in face.items():
        m = (nout == 1) & (low[:, d] if side == 0 else high[:, d])
        if not np.any(m):
            continue
        cells = G[m]
        t = f["type"]
        if t == "zero":
            add_zero(cells)
        elif t in ("circular", "symmetric"):
            src = cells.copy()
            src[:, d] = fmap(cells[:, d], int(n[d]), t)
            add_unit(cells, b, src)
        elif t == "halo":
            sets.append(_halo_rows(b, blocks, d, side, f, cells, comps))
        elif t == "csr":
            sets.append(_face_csr_rows(b, blk, d, side, f, cells, comps))
        else:
            raise OracleError(f"unknown face type {t}")
    return concat_rowsets(sets)


def _depth_along(cells, n, d, side):
    """Depth ``r`` (0 next to the data) and along index of face ghosts of a
    2-D block."""
    r = (-cells[:, d] - 1) if side == 0 else (cells[:, d] - n[d])
    return r, cells[:, 1 - d]


def _halo_rows(b, blocks, d, side, f, cells, comps):
    """Halo copy across a block edge (Sec. III-B, ``A_ij = delta_ij``): the
    ghost at depth r and along index s reads the source block's data at depth
    r behind its own edge, along index s (or ``len - 1 - s`` when flipped)."""
    n = np.asarray(blocks[b]["n"], np.int64)
    if blocks[b]["n"][2] != 1:
        raise OracleError("halo faces are defined for 2-D blocks")
    sb, sa, ss = f["src_block"], f["src_axis"], f["src_side"]
    sn = np.asarray(blocks[sb]["n"], np.int64)
    ln = int(n[1 - d])
    if int(sn[1 - sa]) != ln:
        raise OracleError("halo edge lengths differ")
    r, s = _depth_along(cells, n, d, side)
    if f["flip"]:
        s = ln - 1 - s
    src = np.zeros_like(cells)
    src[:, sa] = r if ss == 0 else sn[sa] - 1 - r
    src[:, 1 - sa] = s
    cc, ijk = _comps_cells(comps, cells)
    return unit_rowset(b, cc, ijk, sb, cc, np.tile(src, (len(comps), 1)))


def _face_csr_rows(b, blk, d, side, f, cells, comps):
    """A face given as user CSR rows: row (r, s) reads data layers
    ``layers[r, s, :nnz]`` behind the face, at the same along index."""
    n = np.asarray(blk["n"], np.int64)
    r, s = _depth_along(cells, n, d, side)
    nnz = np.asarray(f["nnz"], np.int64)[r, s]
    lay = np.asarray(f["layers"], np.int64)[r, s]
    wts = np.asarray(f["weights"], np.float64)[r, s]
    R = len(cells)
    mask = np.arange(lay.shape[1])[None, :] < nnz[:, None]
    e_row = np.repeat(np.arange(R, dtype=np.int64), nnz)
    e_lay = lay[mask]
    e_w = wts[mask]
    src = np.zeros((len(e_row), 3), np.int64)
    src[:, d] = e_lay if side == 0 else n[d] - 1 - e_lay
    src[:, 1 - d] = s[e_row]
    sets = []
    for c in comps:
        rs = empty_rowset(b, np.full(R, c), cells)
        rs["e_row"] = e_row.copy()
        rs["e_b"] = np.full(len(e_row), b, np.int64)
        rs["e_c"] = np.full(len(e_row), c, np.int64)
        rs["e_ijk"] = src.copy()
        rs["e_w"] = e_w.copy()
        sets.append(rs)
    return concat_rowsets(sets)
