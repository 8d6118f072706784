"""Seeded synthetic workloads for the ghost-fill operator ``g = A x + b``.

The CUDA path's tests and benchmark and the FP64 oracle both consume what this
module produces.  It holds none of the method's arithmetic: no index maps, no
generated interpolation weights, no basis-change matrices and no matrix
assembly.  It only draws block shapes, boundary-condition *descriptions* (the
basic sub-matrices a user would write down, Sec. IV-A, Table II) and field
values.  One workload, :func:`staggered_interp`, is a user-given ``Itp``: its
description carries the user's own interpolation tables (Lagrange weights
and rotations written out here as input data, as a user of the library would
write them), which both sides then read as given.

Workload dictionary
-------------------
``{"name", "dtype": "f32"|"f64", "blocks": [block...], "bcs": [bc...],
"fields": [ndarray per block]}``

block
    ``{"n": (n0, n1, n2), "h": (h0, h1, h2), "nlevels": L, "ncomp": C}``.
    Axis 0 is the fastest.  2-D blocks have ``n2 = 1, h2 = 0``.  The data
    region is ``[0, n_d)`` per axis, the full region ``[-h_d, n_d + h_d)``
    (Sec. III-A: ``R_D`` and ``R_F``).
field
    One array per block of shape ``(C, L, n2 + 2 h2, n1 + 2 h1, n0 + 2 h0)``,
    i.e. each component is stored level-major.  Data cells hold the sampled
    values; ghost cells are pre-filled with a quiet NaN so that any read of a
    ghost shows up in the result.

bc kinds (the descriptions; each side turns them into rows on its own)
    ``zero``   ``{block, lo, hi, comps}`` explicit box of ghost cells.
    ``const``  ``{block, lo, hi, comps, values[ncomp_sel, box_volume]}``.
    ``map``    ``{block, lo, hi, comps, src_block, perm, sign, offset}``:
               the source cell of ghost ``g`` is
               ``src[d] = sign[d] * g[perm[d]] + offset[d]`` (``|sign| > 1``
               injects from a finer grid).
    ``csr``    ``{block, lo, hi, comps, row_ptr, col_block, col_comp,
               col_ijk[nnz, 3], val[nnz], rhs[nrows] | None}``; row order is
               comp-major, then the box cells with axis 0 fastest.  A row is
               applied at every level and reads the same level.
    ``faces``  ``{block, corners: "zero"|"product", faces: [face...]}`` with
               face ``{axis, side: 0 (low) | 1 (high), type, ...}`` and type
               one of ``zero``, ``circular``, ``symmetric``, ``halo``
               (``src_block, src_axis, src_side, flip``) or ``csr``
               (``nnz[h, len], layers[h, len, 8], weights[h, len, 8]``, row
               ``(r, s)`` = depth ``r`` from the data, along index ``s``).
    ``cubed_sphere_edges``  ``{panels[6], N, h, p, scalar_comps,
               vector_pair | None}``: panel-edge sync of six equiangular
               gnomonic panels by ``p``-point interpolation along the
               neighbour row, with the ``vector_pair`` components rotated.
    ``sync``   block-edge averaging (``Sync`` of Sec. III-B): the fields of
               ``csr`` with the box inside the *data* region; the rows
               overwrite those data cells.
"""
from __future__ import annotations

import math

import numpy as np

DTYPES = {"f32": np.float32, "f64": np.float64}


# ----------------------------------------------------------------------------
# generic helpers
# ----------------------------------------------------------------------------
def block2d(nx, ny, h, nlevels=1, ncomp=1):
    return {"n": (int(nx), int(ny), 1), "h": (int(h), int(h), 0),
            "nlevels": int(nlevels), "ncomp": int(ncomp)}


def block3d(n, h, nlevels=1, ncomp=1):
    return {"n": (int(n[0]), int(n[1]), int(n[2])),
            "h": (int(h), int(h), int(h)), "nlevels": int(nlevels),
            "ncomp": int(ncomp)}


def full_shape(blk):
    n, h = blk["n"], blk["h"]
    return (blk["ncomp"], blk["nlevels"], n[2] + 2 * h[2], n[1] + 2 * h[1],
            n[0] + 2 * h[0])


def data_view(arr, blk):
    """The data region ``R_D`` of one block's field array (a view)."""
    h, n = blk["h"], blk["n"]
    return arr[:, :, h[2]:h[2] + n[2], h[1]:h[1] + n[1], h[0]:h[0] + n[0]]


def empty_fields(blocks, dtype):
    out = []
    for blk in blocks:
        a = np.empty(full_shape(blk), dtype=DTYPES[dtype])
        a.fill(np.nan)
        out.append(a)
    return out


def uniform_fields(blocks, dtype, lo, hi, seed):
    rng = np.random.default_rng(seed)
    fields = empty_fields(blocks, dtype)
    for blk, a in zip(blocks, fields):
        d = data_view(a, blk)
        d[...] = rng.uniform(lo, hi, size=d.shape)
    return fields


def dirichlet_udf(i, j, comp, t):
    """A pure function of the ghost cell, the component and the time, with
    dyadic coefficients so that FP32 and FP64 evaluations are exact: the
    boundary values of a time-dependent Dirichlet problem."""
    return 0.25 * i - 0.5 * j + 0.125 * t + comp


def dirichlet_block(nx=20, ny=14, h=2, nlevels=3, ncomp=2, dtype="f64", t=0.0, seed=21):
    """One 2-D block whose ghost boxes (four faces, four corners) are
    pure-function boundaries ``b = dirichlet_udf(i, j, comp, t)`` (BC_CONST
    tables, Sec. III-B), data uniform in [-1, 1]."""
    blk = block2d(nx, ny, h, nlevels, ncomp)
    fields = uniform_fields([blk], dtype, -1.0, 1.0, seed)
    comps = list(range(ncomp))
    bcs = []
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            if a == 0 and b == 0:
                continue
            lo = [-h if a < 0 else (nx if a > 0 else 0), -h if b < 0 else (ny if b > 0 else 0), 0]
            hi = [0 if a < 0 else (nx + h if a > 0 else nx), 0 if b < 0 else (ny + h if b > 0 else ny), 1]
            jj, ii = np.meshgrid(np.arange(lo[1], hi[1]), np.arange(lo[0], hi[0]), indexing="ij")
            vals = np.concatenate([dirichlet_udf(ii.ravel(), jj.ravel(), c, t) for c in comps])
            bcs.append({"kind": "const", "block": 0, "lo": tuple(lo), "hi": tuple(hi),
                        "comps": comps, "values": vals.astype(np.float64)})
    return {"name": f"dirichlet{nx}x{ny}_h{h}_t{t}", "dtype": dtype, "blocks": [blk],
            "bcs": bcs, "fields": fields}


def ghost_on_ghost(sizes=((12, 9), (7, 10)), h=3, nlevels=2, ncomp=2, dtype="f64",
                   seed=22, scheme="extrapolate", sweeps=3):
    """2-D blocks whose faces are user CSR rows that read other ghost values
    (the iterative form of Sec. II-B, resolved by ``sweeps`` Jacobi sweeps
    from zero ghosts); corners zero.

    ``scheme``: ``"extrapolate"`` -- the ghost at depth r is
    ``2 v(r-1) - v(r-2)``, v(-1), v(-2) the first two data layers behind the
    face and v(r >= 0) the ghosts (exact linear extrapolation after h
    sweeps); ``"smooth"`` -- ``0.5 data(layer r) + 0.2 (g(r, s-1) + g(r, s+1))
    + 0.1 g(r-1, s)`` (the neighbours along the face wrap round; g(-1) is
    data layer 0) plus b = 0.05, a contraction with ghost cycles."""
    blocks = [block2d(nx, ny, h, nlevels, ncomp) for nx, ny in sizes]
    fields = uniform_fields(blocks, dtype, -1.0, 1.0, seed)
    comps = list(range(ncomp))
    bcs = []
    for b, blk in enumerate(blocks):
        n = blk["n"]
        for d in (0, 1):
            for side in (0, 1):
                ln = n[1 - d]

                def cell(q, s_, d=d, side=side, n=n):
                    # q < 0: data layer -1 - q behind the face; q >= 0: ghost depth q
                    ijk = [0, 0, 0]
                    if q < 0:
                        L = -1 - q
                        ijk[d] = L if side == 0 else n[d] - 1 - L
                    else:
                        ijk[d] = -1 - q if side == 0 else n[d] + q
                    ijk[1 - d] = s_
                    return ijk
                lo, hi = [0, 0, 0], [n[0], n[1], 1]
                lo[d], hi[d] = (-h, 0) if side == 0 else (n[d], n[d] + h)
                # box cells in box order (axis 0 fastest)
                box = [(i, j) for j in range(lo[1], hi[1]) for i in range(lo[0], hi[0])]
                ents = []
                for (i, j) in box:
                    g = (i, j)
                    r = (-1 - g[d]) if side == 0 else (g[d] - n[d])
                    s_ = g[1 - d]
                    if scheme == "extrapolate":
                        ents.append([(cell(r - 1, s_), 2.0), (cell(r - 2, s_), -1.0)])
                    elif scheme == "smooth":
                        e = [(cell(-1 - r, s_) if r < n[d] else cell(-1, s_), 0.5),
                             (cell(r, (s_ - 1) % ln), 0.2), (cell(r, (s_ + 1) % ln), 0.2),
                             (cell(r - 1, s_), 0.1)]
                        ents.append(e)
                    else:
                        raise ValueError(scheme)
                nnz = np.array([len(e) for e in ents] * len(comps), np.int64)
                rp = np.concatenate([[0], np.cumsum(nnz)])
                col_ijk = np.array([c for _ in comps for e in ents for c, _w in e], np.int32)
                val = np.array([w_ for _ in comps for e in ents for _c, w_ in e], np.float64)
                col_comp = np.array([c for c in comps for e in ents for _ in e], np.int32)
                rhs = None
                if scheme == "smooth":
                    rhs = np.full(len(box) * len(comps), 0.05)
                bcs.append({"kind": "csr", "block": b, "lo": tuple(lo), "hi": tuple(hi),
                            "comps": comps, "row_ptr": rp.astype(np.int64),
                            "col_block": np.full(len(val), b, np.int32), "col_comp": col_comp,
                            "col_ijk": col_ijk.reshape(-1, 3), "val": val, "rhs": rhs})
        # corners zero
        for a in (-1, 1):
            for c in (-1, 1):
                lo = [-h if a < 0 else n[0], -h if c < 0 else n[1], 0]
                hi = [0 if a < 0 else n[0] + h, 0 if c < 0 else n[1] + h, 1]
                bcs.append({"kind": "zero", "block": b, "lo": tuple(lo), "hi": tuple(hi),
                            "comps": comps})
    return {"name": f"ghost_on_ghost_{scheme}_k{sweeps}", "dtype": dtype, "blocks": blocks,
            "bcs": bcs, "fields": fields, "ghost_sweeps": int(sweeps)}


def _lagrange(tau, p):
    w = np.ones(p)
    for k in range(p):
        for m in range(p):
            if m != k:
                w[k] *= (tau - m) / (k - m)
    return w


def swap_xy(w):
    """The same workload with axes 0 and 1 exchanged (blocks, boxes, maps,
    tables and fields), so that every stencil steps along the other axis."""
    def sw(t):
        t = list(t)
        return (t[1], t[0]) + tuple(t[2:])
    out = dict(w, name=w["name"] + "_yx")
    out["blocks"] = [dict(b, n=sw(b["n"]), h=sw(b["h"])) for b in w["blocks"]]
    out["fields"] = [np.ascontiguousarray(a.swapaxes(3, 4)) for a in w["fields"]]
    bcs = []
    for bc in w["bcs"]:
        d = dict(bc, lo=sw(bc["lo"]), hi=sw(bc["hi"]))
        if bc["kind"] == "interp":
            # box order is axis 0 fastest: reorder the per-cell tables too
            nx_, ny_ = bc["hi"][0] - bc["lo"][0], bc["hi"][1] - bc["lo"][1]
            order = np.arange(nx_ * ny_).reshape(ny_, nx_).T.reshape(-1)
            st = np.asarray(bc["start"]).reshape(-1, 3)[order]
            d["start"] = st[:, [1, 0, 2]].astype(np.int32)
            d["axis"] = np.asarray(1 - np.asarray(bc["axis"])[order], np.int32)
            d["w"] = np.asarray(bc["w"])[order]
            d["rot"] = np.asarray(bc["rot"])[order]
        elif bc["kind"] == "map":
            perm = list(bc["perm"])
            perm[0], perm[1] = perm[1], perm[0]
            perm = [1 - q if q < 2 else q for q in perm]
            d["perm"], d["sign"], d["offset"] = tuple(perm), sw(bc["sign"]), sw(bc["offset"])
        elif bc["kind"] not in ("zero",):
            raise ValueError(bc["kind"])
        bcs.append(d)
    out["bcs"] = bcs
    return out


def staggered_interp(nx=16, ny=12, h=2, nlevels=3, p=4, dtype="f64", seed=23, rotate=True):
    """Two 2-D blocks side by side along x whose rows are staggered by half a
    cell: each block's ghost columns facing the other are user interpolation
    tables (Sec. III-B ``Itp`` given by the user): the ghost at depth r and
    row s reads the other block's data column at depth r, interpolated along
    y at s +- 1/2 with ``p``-point Lagrange weights (stencil clamped into the
    data).  Components (h, u, v); with ``rotate`` the pair (u, v) is turned
    by a per-cell angle after interpolation.  The y faces are circular, the
    outer x faces and the corners zero."""
    blocks = [block2d(nx, ny, h, nlevels, 3) for _ in range(2)]
    fields = uniform_fields(blocks, dtype, -1.0, 1.0, seed)
    comps = [0, 1, 2]
    bcs = []
    for b in range(2):
        other = 1 - b
        side = 1 if b == 0 else 0          # the face towards the other block
        shift = 0.5 if b == 0 else -0.5
        lo = [nx, 0, 0] if side else [-h, 0, 0]
        hi = [nx + h, ny, 1] if side else [0, ny, 1]
        starts, axes, ws, rots = [], [], [], []
        for j in range(lo[1], hi[1]):
            for i in range(lo[0], hi[0]):
                r = i - nx if side else -1 - i
                t = j + shift
                st = int(np.clip(np.floor(t) - (p // 2 - 1), 0, ny - p))
                src_i = r if side else nx - 1 - r
                starts.append((src_i, st, 0))
                axes.append(1)
                ws.append(_lagrange(t - st, p))
                th = 0.05 * (j + 1) * (r + 1) if rotate else 0.0
                rots.append((np.cos(th), -np.sin(th), np.sin(th), np.cos(th)))
        bcs.append({"kind": "interp", "block": b, "lo": tuple(lo), "hi": tuple(hi),
                    "comps": comps, "src_block": other, "p": p,
                    "start": np.array(starts, np.int32), "axis": np.array(axes, np.int32),
                    "w": np.array(ws, np.float64), "rot_comp": (1, 2),
                    "rot": np.array(rots, np.float64)})
        # outer x face zero, y faces circular, corners zero
        olo = [-h, 0, 0] if side else [nx, 0, 0]
        ohi = [0, ny, 1] if side else [nx + h, ny, 1]
        bcs.append({"kind": "zero", "block": b, "lo": tuple(olo), "hi": tuple(ohi),
                    "comps": comps})
        for yside in (0, 1):
            ylo = [0, -h, 0] if yside == 0 else [0, ny, 0]
            yhi = [nx, 0, 1] if yside == 0 else [nx, ny + h, 1]
            off = ny if yside == 0 else -ny
            bcs.append({"kind": "map", "block": b, "lo": tuple(ylo), "hi": tuple(yhi),
                        "comps": comps, "src_block": b, "perm": (0, 1, 2), "sign": (1, 1, 1),
                        "offset": (0, off, 0)})
        for a in (-1, 1):
            for c in (-1, 1):
                clo = [-h if a < 0 else nx, -h if c < 0 else ny, 0]
                chi = [0 if a < 0 else nx + h, 0 if c < 0 else ny + h, 1]
                bcs.append({"kind": "zero", "block": b, "lo": tuple(clo), "hi": tuple(chi),
                            "comps": comps})
    return {"name": f"staggered_interp{nx}x{ny}_p{p}", "dtype": dtype, "blocks": blocks,
            "bcs": bcs, "fields": fields}


def total_full_values(w):
    return sum(int(np.prod(full_shape(b))) for b in w["blocks"])


# ----------------------------------------------------------------------------
# Algorithm 1: three 5x5 blocks, the right ghost of block 1 is a rotated copy
# of block 2, the left ghost a user CSR from block 0, the rest zero.
# ----------------------------------------------------------------------------
def alg1_example(seed=11, dtype="f64"):
    """The worked example of Alg. 1 (three blocks, data 5x5, full 7x7).

    The paper's grid index ``[block, idx1, idx2]`` maps onto this layout as
    ``idx2 -> axis 0 (i)`` and ``idx1 -> axis 1 (j)``.  The printed column of
    the right-ghost iterator, ``(2, 9 - idx2, idx1)``, therefore reads block 2
    at ``i' = j, j' = 9 - i``.
    """
    rng = np.random.default_rng(seed)
    blocks = [block2d(5, 5, 1) for _ in range(3)]
    bcs = []
    # right ghost column of block 1: i = 5, j in [0, 5)
    bcs.append({"kind": "map", "block": 1, "lo": (5, 0, 0), "hi": (6, 5, 1),
                "comps": [0], "src_block": 2, "perm": (1, 0, 2),
                "sign": (1, -1, 1), "offset": (0, 9, 0)})
    # left ghost column of block 1: i = -1, j in [0, 5); a user CSR that reads
    # the two right-most data columns of block 0 (3 entries per row)
    row_ptr, cb, cc, cijk, val = [0], [], [], [], []
    for j in range(5):
        jj = sorted(rng.choice(5, size=2, replace=False).tolist())
        cols = [(4, j), (3, jj[0]), (4, jj[1])]
        w = rng.uniform(0.1, 1.0, size=3)
        w = w / w.sum()
        for (ci, cj), wv in zip(cols, w):
            cb.append(0)
            cc.append(0)
            cijk.append((ci, cj, 0))
            val.append(float(wv))
        row_ptr.append(len(val))
    bcs.append({"kind": "csr", "block": 1, "lo": (-1, 0, 0), "hi": (0, 5, 1),
                "comps": [0], "row_ptr": np.array(row_ptr, np.int64),
                "col_block": np.array(cb, np.int32),
                "col_comp": np.array(cc, np.int32),
                "col_ijk": np.array(cijk, np.int32).reshape(-1, 3),
                "val": np.array(val, np.float64), "rhs": None})
    # zero: bottom and top ghost rows of block 1, corners included
    bcs.append({"kind": "zero", "block": 1, "lo": (-1, -1, 0),
                "hi": (6, 0, 1), "comps": [0]})
    bcs.append({"kind": "zero", "block": 1, "lo": (-1, 5, 0),
                "hi": (6, 6, 1), "comps": [0]})
    fields = uniform_fields(blocks, dtype, -1.0, 1.0, seed + 1)
    return {"name": "alg1", "dtype": dtype, "blocks": blocks, "bcs": bcs,
            "fields": fields}


# ----------------------------------------------------------------------------
# HPCG-like single 3-D block with face boundary conditions
# ----------------------------------------------------------------------------
def hpcg_block(n=128, variant="Z", seed=2, dtype="f64", nblocks=1):
    """A 3-D block (or ``nblocks`` independent copies) with h = 1.

    Variants: ``Z`` all six faces zero; ``P`` x faces circular (periodic),
    other faces zero; ``S`` y faces symmetric, other faces zero.  Edge and
    corner ghosts follow the per-axis product rule (``corners="product"``).
    """
    nn = (n, n, n) if np.isscalar(n) else tuple(n)
    blocks = [block3d(nn, 1) for _ in range(nblocks)]
    bcs = []
    for b in range(nblocks):
        faces = []
        for axis in range(3):
            for side in (0, 1):
                t = "zero"
                if variant == "P" and axis == 0:
                    t = "circular"
                if variant == "S" and axis == 1:
                    t = "symmetric"
                faces.append({"axis": axis, "side": side, "type": t})
        bcs.append({"kind": "faces", "block": b, "corners": "product",
                    "faces": faces})
    fields = uniform_fields(blocks, dtype, 0.0, 1.0, seed)
    return {"name": f"hpcg{nn[0]}_{variant}x{nblocks}", "dtype": dtype,
            "blocks": blocks, "bcs": bcs, "fields": fields}


# ----------------------------------------------------------------------------
# Many uneven 2-D blocks, one drawn boundary condition per edge
# ----------------------------------------------------------------------------
FACE_TYPES = ("halo", "circular", "symmetric", "zero", "csr")


def _edge_len(blk, axis):
    return blk["n"][1 - axis]


def batching(nblocks=512, side_lo=16, side_hi=256, lev_lo=1, lev_hi=64, h=2,
             seed=4, dtype="f32"):
    """``nblocks`` 2-D blocks, sides log-uniform in [side_lo, side_hi],
    levels uniform in [lev_lo, lev_hi], fields uniform in [-1, 1].  Each edge
    draws its boundary type uniformly from :data:`FACE_TYPES`; a halo edge
    copies from a random edge (of any block) with the same length and level
    count, orientation flip drawn, redrawn as another type if no such edge
    exists.  A CSR edge draws 2..8 distinct data layers out of the first 8
    behind the edge, weights in (0, 1] summing to one.  Corners are zero as in
    Alg. 1.
    """
    rng = np.random.default_rng(seed)
    lg = rng.uniform(math.log(side_lo), math.log(side_hi + 1), size=(nblocks, 2))
    sides = np.minimum(np.floor(np.exp(lg)).astype(int), side_hi)
    levels = rng.integers(lev_lo, lev_hi + 1, size=nblocks)
    blocks = [block2d(sides[b, 0], sides[b, 1], h, levels[b])
              for b in range(nblocks)]
    # index of edges by (length, levels) for halo partners
    by_key = {}
    for b, blk in enumerate(blocks):
        for axis in (0, 1):
            for side in (0, 1):
                key = (_edge_len(blk, axis), blk["nlevels"])
                by_key.setdefault(key, []).append((b, axis, side))
    bcs = []
    for b, blk in enumerate(blocks):
        faces = []
        for axis in (0, 1):
            for side in (0, 1):
                ln = _edge_len(blk, axis)
                nnorm = blk["n"][axis]
                while True:
                    t = FACE_TYPES[int(rng.integers(len(FACE_TYPES)))]
                    if t in ("circular", "symmetric") and h > nnorm:
                        continue
                    if t == "halo":
                        cand = [e for e in by_key[(ln, blk["nlevels"])]
                                if e != (b, axis, side)
                                and blocks[e[0]]["n"][e[1]] >= h]
                        if not cand:
                            continue
                        sb, sa, ss = cand[int(rng.integers(len(cand)))]
                        faces.append({"axis": axis, "side": side, "type": t,
                                      "src_block": int(sb), "src_axis": int(sa),
                                      "src_side": int(ss),
                                      "flip": int(rng.integers(2))})
                    elif t == "csr":
                        depth = min(8, nnorm)
                        nnz = rng.integers(2, 9, size=(h, ln))
                        nnz = np.minimum(nnz, depth)
                        layers = np.zeros((h, ln, 8), np.int32)
                        weights = np.zeros((h, ln, 8), np.float64)
                        for r in range(h):
                            for s in range(ln):
                                k = int(nnz[r, s])
                                layers[r, s, :k] = np.sort(
                                    rng.choice(depth, size=k, replace=False))
                                w = 1.0 - rng.random(k)   # (0, 1]
                                weights[r, s, :k] = w / w.sum()
                        faces.append({"axis": axis, "side": side, "type": t,
                                      "nnz": nnz.astype(np.int32),
                                      "layers": layers, "weights": weights})
                    else:
                        faces.append({"axis": axis, "side": side, "type": t})
                    break
        bcs.append({"kind": "faces", "block": b, "corners": "zero",
                    "faces": faces})
    fields = uniform_fields(blocks, dtype, -1.0, 1.0, seed + 100)
    return {"name": f"batching{nblocks}", "dtype": dtype, "blocks": blocks,
            "bcs": bcs, "fields": fields}


# ----------------------------------------------------------------------------
# Cubed sphere: field synthesis only (equiangular gnomonic panels)
# ----------------------------------------------------------------------------
def _panel_xyz(panel, a, b):
    """Cube-surface point of equiangular coordinates (a, b) on ``panel``
    (panels 0..3 around the equator facing +X, +Y, -X, -Y; 4 = +Z, 5 = -Z).
    Used here only to synthesise smooth fields."""
    x, y = np.tan(a), np.tan(b)
    one = np.ones_like(x)
    table = {
        0: (one, x, y), 1: (-x, one, y), 2: (-one, -x, y), 3: (x, -one, y),
        4: (-y, x, one), 5: (y, x, -one),
    }
    X, Y, Z = table[panel]
    r = np.sqrt(X * X + Y * Y + Z * Z)
    return X / r, Y / r, Z / r


def cell_angle(N, idx):
    return -math.pi / 4 + (np.asarray(idx, np.float64) + 0.5) * (math.pi / (2 * N))


def smooth_sphere_scalar(rng, degree=16, nterms=48):
    """A random polynomial of total degree <= ``degree`` in (X, Y, Z), written
    as a sum of ridge terms ``c (u . r)^d``; restricted to the sphere it lies
    in the span of the spherical harmonics of degree <= ``degree``.  Returns a
    callable on unit vectors."""
    dirs = rng.normal(size=(nterms, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    degs = rng.integers(0, degree + 1, size=nterms)
    coef = rng.normal(size=nterms) / (1.0 + degs) ** 2

    def f(X, Y, Z):
        out = np.zeros_like(X)
        for u, d, c in zip(dirs, degs, coef):
            out += c * (u[0] * X + u[1] * Y + u[2] * Z) ** int(d)
        return out
    return f


def rigid_rotation_covariant(panel, a, b, axis, speed, step=1e-6):
    """Covariant components ``(V . dr/da, V . dr/db)`` of the rigid-rotation
    wind ``V = speed * (axis x r)`` on the unit sphere, the derivatives of the
    unit position taken by central differences (a field synthesiser, not the
    method's basis)."""
    X, Y, Z = _panel_xyz(panel, a, b)
    ax = np.asarray(axis, np.float64)
    VX = speed * (ax[1] * Z - ax[2] * Y)
    VY = speed * (ax[2] * X - ax[0] * Z)
    VZ = speed * (ax[0] * Y - ax[1] * X)
    pa = _panel_xyz(panel, a + step, b)
    ma = _panel_xyz(panel, a - step, b)
    pb = _panel_xyz(panel, a, b + step)
    mb = _panel_xyz(panel, a, b - step)
    ea = [(p - m) / (2 * step) for p, m in zip(pa, ma)]
    eb = [(p - m) / (2 * step) for p, m in zip(pb, mb)]
    ua = VX * ea[0] + VY * ea[1] + VZ * ea[2]
    ub = VX * eb[0] + VY * eb[1] + VZ * eb[2]
    return ua, ub


def _corner_csr(N, h, panel, corner, ncomp, scalar_comps, vector_pair):
    """User CSR for the h x h corner ghosts of ``panel`` at ``corner``
    (0: low-low, 1: high-low, 2: low-high, 3: high-high in (i, j)).

    Scalar components: weight 1/3 on each of the three data cells that touch
    the cube vertex (this panel's corner cell and the two other panels'
    corner cells nearest the vertex).  Vector components: a unit copy of this
    panel's own corner cell (no rotation)."""
    ci = 0 if corner in (0, 2) else N - 1
    cj = 0 if corner in (0, 1) else N - 1
    a, b = cell_angle(N, ci), cell_angle(N, cj)
    v = np.array(_panel_xyz(panel, np.float64(a), np.float64(b)))
    vert = np.sign(v)
    touching = [(panel, ci, cj)]
    for q in range(6):
        if q == panel:
            continue
        for qi in (0, N - 1):
            for qj in (0, N - 1):
                w = np.array(_panel_xyz(q, np.float64(cell_angle(N, qi)),
                                        np.float64(cell_angle(N, qj))))
                if np.all(np.sign(w) == vert):
                    touching.append((q, qi, qj))
    assert len(touching) == 3, touching
    lo_i = -h if corner in (0, 2) else N
    lo_j = -h if corner in (0, 1) else N
    comps = list(scalar_comps) + (list(vector_pair) if vector_pair else [])
    row_ptr, cb, cc, cijk, val = [0], [], [], [], []
    for c in comps:
        for jj in range(lo_j, lo_j + h):
            for ii in range(lo_i, lo_i + h):
                if c in scalar_comps:
                    for (q, qi, qj) in touching:
                        cb.append(q)
                        cc.append(c)
                        cijk.append((qi, qj, 0))
                        val.append(1.0 / 3.0)
                else:
                    cb.append(panel)
                    cc.append(c)
                    cijk.append((ci, cj, 0))
                    val.append(1.0)
                row_ptr.append(len(val))
    return {"kind": "csr", "block": panel, "lo": (lo_i, lo_j, 0),
            "hi": (lo_i + h, lo_j + h, 1), "comps": comps,
            "row_ptr": np.array(row_ptr, np.int64),
            "col_block": np.array(cb, np.int32),
            "col_comp": np.array(cc, np.int32),
            "col_ijk": np.array(cijk, np.int32).reshape(-1, 3),
            "val": np.array(val, np.float64), "rhs": None}


def cubed_sphere(N=32, h=2, p=4, nlevels=1, fields=("scalar",), dtype="f64",
                 seed=1, quad=None, centred=False, sweeps=10):
    """Six equiangular gnomonic panels of N x N cells with halo h.

    ``quad = nq`` asks for reconstruction-and-quadrature edge rows (each
    edge ghost the average of nq x nq Gauss points, each point reconstructed
    from a p x p patch of the neighbour panel, Sec. II-B) instead of the 1-D
    Lagrange rows along the neighbour row.  ``centred`` (with ``quad``)
    keeps every patch centred on its ghost, so that patches take ghost cells
    of the neighbour panel (HOPE's iterative form, Sec. II-B), resolved by
    ``sweeps`` Jacobi sweeps (the workload's ``ghost_sweeps``).

    ``fields`` is ``("scalar",)`` (one component uniform in [-1, 1]) or
    ``("h", "u", "v")`` (a smooth height field of 1e4 +- 100 m built from a
    degree-16 polynomial on the sphere, and covariant rigid-rotation wind
    components of 50 m/s about a seeded axis, one axis and scaling per
    level).  Corner ghosts are filled by user CSR rows (see
    :func:`_corner_csr`)."""
    rng = np.random.default_rng(seed)
    ncomp = len(fields)
    blocks = [block2d(N, N, h, nlevels, ncomp) for _ in range(6)]
    arrs = empty_fields(blocks, dtype)
    idx = np.arange(N)
    a = cell_angle(N, idx)[None, :]
    b = cell_angle(N, idx)[:, None]
    A, B = np.broadcast_arrays(a, b)
    if fields == ("scalar",):
        for pnl in range(6):
            d = data_view(arrs[pnl], blocks[pnl])
            d[...] = rng.uniform(-1.0, 1.0, size=d.shape)
        scalar_comps, vpair = [0], None
    elif tuple(fields) == ("h", "u", "v"):
        poly = smooth_sphere_scalar(rng)
        pts = [_panel_xyz(pnl, A, B) for pnl in range(6)]
        vals = [poly(*pt) for pt in pts]
        pmax = max(float(np.abs(v).max()) for v in vals) or 1.0
        lev_scale = rng.uniform(0.5, 1.0, size=nlevels)
        lev_shift = rng.uniform(-20.0, 20.0, size=nlevels)
        axes = rng.normal(size=(nlevels, 3))
        axes /= np.linalg.norm(axes, axis=1, keepdims=True)
        for pnl in range(6):
            d = data_view(arrs[pnl], blocks[pnl])
            base = vals[pnl] / pmax
            for lev in range(nlevels):
                d[0, lev, 0] = 1e4 + lev_shift[lev] + 80.0 * lev_scale[lev] * base
                ua, ub = rigid_rotation_covariant(pnl, A, B, axes[lev], 50.0)
                d[1, lev, 0] = ua
                d[2, lev, 0] = ub
        scalar_comps, vpair = [0], [1, 2]
    else:
        raise ValueError(fields)
    bcs = [{"kind": "cubed_sphere_edges", "panels": list(range(6)), "N": N,
            "h": h, "p": p, "scalar_comps": scalar_comps,
            "vector_pair": vpair}]
    if quad:
        bcs[0]["quad"] = int(quad)
        if centred:
            bcs[0]["centred"] = True
    for pnl in range(6):
        for corner in range(4):
            bcs.append(_corner_csr(N, h, pnl, corner, ncomp, scalar_comps,
                                   vpair))
    qtag = (f"_q{int(quad)}" + (f"c{int(sweeps)}" if centred else "")) if quad else ""
    w = {"name": f"cubed_sphere{N}_h{h}_p{p}{qtag}_L{nlevels}", "dtype": dtype,
         "blocks": blocks, "bcs": bcs, "fields": arrs,
         "sphere": {"N": N, "h": h, "p": p, "quad": quad, "fields": tuple(fields)}}
    if quad and centred:
        w["ghost_sweeps"] = int(sweeps)
    return w


# ----------------------------------------------------------------------------
# The five named workloads
# ----------------------------------------------------------------------------
def tiny_cubed_sphere(seed=1):
    """6 x 32^2, h = 2, one FP64 scalar in [-1, 1], p = 4."""
    return cubed_sphere(32, 2, 4, 1, ("scalar",), "f64", seed)


def swe_cubed_sphere(N=384, nlevels=32, seed=3):
    """6 x 384^2, h = 3, (h, u, v) x 32 levels FP32, p = 6."""
    return cubed_sphere(N, 3, 6, nlevels, ("h", "u", "v"), "f32", seed)


def adjoint_cubed_sphere(N=768, nlevels=32, seed=5):
    """6 x 768^2, h = 3, (h, u, v) x 32 levels FP32, p = 6."""
    return cubed_sphere(N, 3, 6, nlevels, ("h", "u", "v"), "f32", seed)


def hope_cubed_sphere(N=384, nlevels=32, seed=3):
    """6 x 384^2, h = 3, (h, u, v) x 32 levels FP32; every edge ghost the
    2 x 2 Gauss-point average of a 4 x 4 tensor-product reconstruction on the
    neighbour panel (16 entries per scalar row, 32 per vector row)."""
    return cubed_sphere(N, 3, 4, nlevels, ("h", "u", "v"), "f32", seed, quad=2)


def cotangent_like(w, seed):
    """A random cotangent over the full region of every block, U[-1, 1]
    everywhere (ghost cells included)."""
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1.0, 1.0, size=a.shape).astype(a.dtype)
            for a in w["fields"]]


def copy_fields(w):
    return [a.copy() for a in w["fields"]]


# ----------------------------------------------------------------------------
# block-edge averaging: node-centred blocks that share their edge nodes
# ----------------------------------------------------------------------------
def sync_grid(bx=3, by=3, n=17, h=2, nlevels=4, ncomp=2, dtype="f64", seed=12):
    """``bx`` x ``by`` node-centred 2-D blocks of ``n`` x ``n`` nodes; block
    ``(a, b)`` holds the global nodes ``(a (n-1) + i, b (n-1) + j)``, so
    neighbouring blocks store their common edge twice (corner nodes up to
    four times), as in multi-block MCV grids.  Boundary descriptions:

    * ``sync`` rows on every stored copy of a shared node: the mean of all
      copies (weights ``1/k`` over the ``k`` copies, all components alike);
    * ghost layers: a ``map`` from the neighbouring block across each inner
      edge, skipping the shared node line (ghost depth ``r`` reads the
      neighbour's node ``1 + r`` behind the edge); ``zero`` on the outer
      boundary and on the corners.

    Fields are uniform in [-1, 1] (so the copies of a node differ).
    """
    rng_blocks = [block2d(n, n, h, nlevels, ncomp) for _ in range(bx * by)]
    bid = lambda a, b: b * bx + a  # noqa: E731
    # copies of every node
    copies = {}
    for b in range(by):
        for a in range(bx):
            for j in range(n):
                for i in range(n):
                    X, Y = a * (n - 1) + i, b * (n - 1) + j
                    copies.setdefault((X, Y), []).append((bid(a, b), i, j))
    bcs = []
    comps = list(range(ncomp))
    for b in range(by):
        for a in range(bx):
            k = bid(a, b)
            # shared nodes of this block, as boxes: the shared columns, then
            # the rest of the shared rows
            boxes = []
            cols = [i for i, on in ((0, a > 0), (n - 1, a < bx - 1)) if on]
            for i in cols:
                boxes.append(((i, 0, 0), (i + 1, n, 1)))
            i_lo = 1 if 0 in cols else 0
            i_hi = n - 1 if (n - 1) in cols else n
            for j, on in ((0, b > 0), (n - 1, b < by - 1)):
                if on and i_hi > i_lo:
                    boxes.append(((i_lo, j, 0), (i_hi, j + 1, 1)))
            for lo, hi in boxes:
                cells = [(i, j) for j in range(lo[1], hi[1]) for i in range(lo[0], hi[0])]
                row_ptr, cb, cc, cijk, val = [0], [], [], [], []
                for c in comps:
                    for i, j in cells:
                        grp = copies[(a * (n - 1) + i, b * (n - 1) + j)]
                        for (ob, oi, oj) in grp:
                            cb.append(ob)
                            cc.append(c)
                            cijk.append((oi, oj, 0))
                            val.append(1.0 / len(grp))
                        row_ptr.append(len(val))
                bcs.append({"kind": "sync", "block": k, "lo": lo, "hi": hi,
                            "comps": comps,
                            "row_ptr": np.array(row_ptr, np.int64),
                            "col_block": np.array(cb, np.int32),
                            "col_comp": np.array(cc, np.int32),
                            "col_ijk": np.array(cijk, np.int32).reshape(-1, 3),
                            "val": np.array(val, np.float64), "rhs": None})
            # ghost layers
            for axis in (0, 1):
                for side in (0, 1):
                    lo = [0, 0, 0]
                    hi = [n, n, 1]
                    lo[axis], hi[axis] = (-h, 0) if side == 0 else (n, n + h)
                    na = a + (1 if side else -1) if axis == 0 else a
                    nb = b + (1 if side else -1) if axis == 1 else b
                    if 0 <= na < bx and 0 <= nb < by:
                        off = [0, 0, 0]
                        off[axis] = (n - 1) if side == 0 else -(n - 1)
                        bcs.append({"kind": "map", "block": k, "lo": tuple(lo),
                                    "hi": tuple(hi), "comps": comps,
                                    "src_block": bid(na, nb), "perm": (0, 1, 2),
                                    "sign": (1, 1, 1), "offset": tuple(off)})
                    else:
                        bcs.append({"kind": "zero", "block": k, "lo": tuple(lo),
                                    "hi": tuple(hi), "comps": comps})
            for cx in ((-h, 0), (n, n + h)):
                for cy in ((-h, 0), (n, n + h)):
                    bcs.append({"kind": "zero", "block": k, "lo": (cx[0], cy[0], 0),
                                "hi": (cx[1], cy[1], 1), "comps": comps})
    fields = uniform_fields(rng_blocks, dtype, -1.0, 1.0, seed)
    return {"name": f"sync{bx}x{by}_n{n}", "dtype": dtype, "blocks": rng_blocks,
            "bcs": bcs, "fields": fields}


# ----------------------------------------------------------------------------
# two grid levels side by side: region steps 1 and 2 (Sec. III-A)
# ----------------------------------------------------------------------------
def two_level(nx=32, ny=24, h=2, nlevels=3, ncomp=1, dtype="f64", seed=13):
    """A fine cell-centred block (``nx`` x ``ny``, step 1) and, to its right,
    a coarse one (``nx/2`` x ``ny/2``, step 2) of one global grid.  The
    coarse block's left ghosts inject the fine cell at the lower-left corner
    of each coarse cell (a ``map`` with scale 2); the fine block's right
    ghosts copy the coarse cell that contains them (``csr`` rows, piecewise
    constant prolongation); every other ghost is zero."""
    assert nx % 2 == 0 and ny % 2 == 0
    fine = block2d(nx, ny, h, nlevels, ncomp)
    coarse = block2d(nx // 2, ny // 2, h, nlevels, ncomp)
    comps = list(range(ncomp))
    bcs = [{"kind": "map", "block": 1, "lo": (-h, 0, 0), "hi": (0, ny // 2, 1),
            "comps": comps, "src_block": 0, "perm": (0, 1, 2), "sign": (2, 2, 1),
            "offset": (nx, 0, 0)}]
    cells = [(i, j) for j in range(ny) for i in range(nx, nx + h)]
    row_ptr, cb, cc, cijk, val = [0], [], [], [], []
    for c in comps:
        for i, j in cells:
            cb.append(1)
            cc.append(c)
            cijk.append(((i - nx) // 2, j // 2, 0))
            val.append(1.0)
            row_ptr.append(len(val))
    bcs.append({"kind": "csr", "block": 0, "lo": (nx, 0, 0), "hi": (nx + h, ny, 1),
                "comps": comps, "row_ptr": np.array(row_ptr, np.int64),
                "col_block": np.array(cb, np.int32), "col_comp": np.array(cc, np.int32),
                "col_ijk": np.array(cijk, np.int32).reshape(-1, 3),
                "val": np.array(val, np.float64), "rhs": None})
    for b, blk in enumerate((fine, coarse)):
        n = blk["n"]
        for axis in (0, 1):
            for side in (0, 1):
                if (b, axis, side) in ((0, 0, 1), (1, 0, 0)):
                    continue
                lo, hi = [0, 0, 0], [n[0], n[1], 1]
                lo[axis], hi[axis] = (-h, 0) if side == 0 else (n[axis], n[axis] + h)
                bcs.append({"kind": "zero", "block": b, "lo": tuple(lo), "hi": tuple(hi),
                            "comps": comps})
        for cx in ((-h, 0), (n[0], n[0] + h)):
            for cy in ((-h, 0), (n[1], n[1] + h)):
                bcs.append({"kind": "zero", "block": b, "lo": (cx[0], cy[0], 0),
                            "hi": (cx[1], cy[1], 1), "comps": comps})
    blocks = [fine, coarse]
    return {"name": f"two_level{nx}x{ny}", "dtype": dtype, "blocks": blocks, "bcs": bcs,
            "fields": uniform_fields(blocks, dtype, -1.0, 1.0, seed)}
