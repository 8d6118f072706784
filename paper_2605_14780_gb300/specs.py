"""Turn boundary-condition descriptions into basic sub-matrices of the C ABI.

Host-side argument construction only: every ghost value is computed by the
CUDA kernels of ``libbcgb300``.  The descriptions are those of
:mod:`paper_2605_14780_gb300.synth` (zero / const / map / csr boxes, per-face
block descriptions and cubed-sphere panel edges); the result is a list of
``bc_submatrix`` dictionaries for :class:`paper_2605_14780_gb300.bc.Plan`.

Face types become index maps (Sec. III-B):

* circular and symmetric faces -- ``fmap`` of the paper, left side
  ``fmap(-x) = x - 1`` (symmetric) or ``N - x`` (circular), right side
  mirrored, written as the affine maps ``i -> -1 - i`` / ``i -> i + N`` on the
  low side and ``i -> 2N - 1 - i`` / ``i -> i - N`` on the high side;
* halo faces -- the ghost at depth r (0 next to the data) and along index s
  reads the source block's data at depth r behind the source edge, along s
  or ``len - 1 - s`` when flipped;
* edges and corners -- zero (``corners="zero"``, as in Alg. 1) or the product
  of the per-axis maps (``corners="product"``), zero as soon as one of the
  faces involved is not a map.
"""
from __future__ import annotations

import itertools

import numpy as np

BC_ZERO, BC_CONST, BC_MAP, BC_INTERP, BC_CSR, BC_SYNC = range(6)
BC_GEOM_USER, BC_GEOM_CUBED_SPHERE, BC_GEOM_CUBED_SPHERE_QUAD = 0, 1, 2
BC_GEOM_CUBED_SPHERE_QUAD_CENTRED = 3


def contiguous_block(blk):
    """C-ABI block descriptor of a contiguous ``(C, L, F2, F1, F0)`` array."""
    n, h = blk["n"], blk["h"]
    F = [n[d] + 2 * h[d] for d in range(3)]
    return {"n": tuple(n), "h": tuple(h), "nlevels": blk["nlevels"],
            "ncomp": blk["ncomp"], "stride": (1, F[0], F[0] * F[1]),
            "level_stride": F[0] * F[1] * F[2]}


def _sub(kind, block, lo, hi, comps, **kw):
    d = {"kind": kind, "block": int(block), "lo": tuple(int(v) for v in lo),
         "hi": tuple(int(v) for v in hi), "comps": [int(c) for c in comps]}
    d.update(kw)
    return d


def _reflect_map(lo_side, N, kind):
    """(sign, offset) of the circular/symmetric map on one side of an axis."""
    if kind == "symmetric":
        return (-1, -1) if lo_side else (-1, 2 * N - 1)
    if kind == "circular":
        return (1, N) if lo_side else (1, -N)
    raise ValueError(kind)


def _check_depth(h, N):
    if h > N:
        raise ValueError(f"ghost depth {h} exceeds the data extent {N}")


def faces_submatrices(bc, blocks):
    b = bc["block"]
    blk = blocks[b]
    n, h = blk["n"], blk["h"]
    comps = list(range(blk["ncomp"]))
    face = {(f["axis"], f["side"]): f for f in bc["faces"]}
    out = []
    ranges = []
    for d in range(3):
        r = [("C", 0, n[d])]
        if h[d] > 0:
            r = [("L", -h[d], 0)] + r + [("H", n[d], n[d] + h[d])]
        ranges.append(r)
    for combo in itertools.product(*ranges):
        outs = [(d, c[0]) for d, c in enumerate(combo) if c[0] != "C"]
        if not outs:
            continue
        lo = [c[1] for c in combo]
        hi = [c[2] for c in combo]
        if len(outs) == 1:
            d, tag = outs[0]
            side = 0 if tag == "L" else 1
            f = face.get((d, side))
            if f is None:
                continue
            out.extend(_face_sub(b, blocks, d, side, f, lo, hi, comps))
            continue
        if bc["corners"] == "zero":
            out.append(_sub(BC_ZERO, b, lo, hi, comps))
            continue
        # product rule
        sign, offset = [1, 1, 1], [0, 0, 0]
        is_map = True
        for d, tag in outs:
            f = face.get((d, 0 if tag == "L" else 1))
            if f is None or f["type"] not in ("circular", "symmetric"):
                is_map = False
                break
            _check_depth(h[d], n[d])
            sign[d], offset[d] = _reflect_map(tag == "L", n[d], f["type"])
        if is_map:
            out.append(_sub(BC_MAP, b, lo, hi, comps, src_block=b,
                            perm=(0, 1, 2), sign=tuple(sign),
                            offset=tuple(offset)))
        else:
            out.append(_sub(BC_ZERO, b, lo, hi, comps))
    return out


def _face_sub(b, blocks, d, side, f, lo, hi, comps):
    blk = blocks[b]
    n = blk["n"]
    t = f["type"]
    if t == "zero":
        return [_sub(BC_ZERO, b, lo, hi, comps)]
    if t in ("circular", "symmetric"):
        _check_depth(blk["h"][d], n[d])
        sign, offset = [1, 1, 1], [0, 0, 0]
        sign[d], offset[d] = _reflect_map(side == 0, n[d], t)
        return [_sub(BC_MAP, b, lo, hi, comps, src_block=b, perm=(0, 1, 2),
                     sign=tuple(sign), offset=tuple(offset))]
    if t == "halo":
        sb, sa, ss = f["src_block"], f["src_axis"], f["src_side"]
        sn = blocks[sb]["n"]
        ln = n[1 - d]
        if sn[1 - sa] != ln:
            raise ValueError("halo edge lengths differ")
        perm, sign, offset = [0, 1, 2], [1, 1, 1], [0, 0, 0]
        # depth r = -1 - g[d] (low side) or g[d] - n[d] (high side)
        perm[sa] = d
        if side == 0:
            rs, ro = -1, -1          # r = -g - 1
        else:
            rs, ro = 1, -n[d]        # r = g - n
        if ss == 0:                  # src[sa] = r
            sign[sa], offset[sa] = rs, ro
        else:                        # src[sa] = sn - 1 - r
            sign[sa], offset[sa] = -rs, sn[sa] - 1 - ro
        perm[1 - sa] = 1 - d
        if f["flip"]:
            sign[1 - sa], offset[1 - sa] = -1, ln - 1
        perm[2], sign[2], offset[2] = 2, 1, 0
        return [_sub(BC_MAP, b, lo, hi, comps, src_block=sb, perm=tuple(perm),
                     sign=tuple(sign), offset=tuple(offset))]
    if t == "csr":
        # rows in box order (axis 0 fastest), per component
        box = [(i, j) for j in range(lo[1], hi[1]) for i in range(lo[0], hi[0])]
        cells = np.array(box, np.int64)
        g = cells[:, d]
        r = (-g - 1) if side == 0 else (g - n[d])
        s = cells[:, 1 - d]
        nnz = np.asarray(f["nnz"], np.int64)[r, s]
        lay = np.asarray(f["layers"], np.int64)[r, s]
        wts = np.asarray(f["weights"], np.float64)[r, s]
        mask = np.arange(lay.shape[1])[None, :] < nnz[:, None]
        e_row = np.repeat(np.arange(len(cells)), nnz)
        e_lay = lay[mask]
        ijk = np.zeros((len(e_row), 3), np.int32)
        ijk[:, d] = e_lay if side == 0 else n[d] - 1 - e_lay
        ijk[:, 1 - d] = s[e_row]
        rp = np.concatenate([[0], np.cumsum(nnz)])
        nc = len(comps)
        row_ptr = np.concatenate([[0]] + [rp[1:] + k * rp[-1] for k in range(nc)])
        return [_sub(BC_CSR, b, lo, hi, comps,
                     row_ptr=row_ptr.astype(np.int64),
                     col_block=np.full(len(e_row) * nc, b, np.int32),
                     col_comp=np.repeat(np.array(comps, np.int32), len(e_row)),
                     col_ijk=np.tile(ijk, (nc, 1)),
                     val=np.tile(wts[mask], nc), rhs=None)]
    raise ValueError(t)


def cubed_sphere_submatrices(bc, blocks):
    N, h, p = bc["N"], bc["h"], bc["p"]
    panels = [int(x) for x in bc["panels"]]
    comps = list(bc["scalar_comps"])
    rot = (-1, -1)
    if bc.get("vector_pair"):
        comps += list(bc["vector_pair"])
        rot = tuple(int(c) for c in bc["vector_pair"])
    out = []
    for P in range(6):
        for d in (0, 1):
            for side in (0, 1):
                lo = [0, 0, 0]
                hi = [N, N, 1]
                lo[d], hi[d] = (-h, 0) if side == 0 else (N, N + h)
                if bc.get("quad"):
                    geom = {"geometry": (BC_GEOM_CUBED_SPHERE_QUAD_CENTRED if bc.get("centred")
                                         else BC_GEOM_CUBED_SPHERE_QUAD),
                            "nquad": int(bc["quad"])}
                else:
                    geom = {"geometry": BC_GEOM_CUBED_SPHERE}
                out.append(_sub(BC_INTERP, panels[P], lo, hi, comps, p=p, rot_comp=rot,
                                cs_panels=tuple(panels), **geom))
    return out


def submatrices(w):
    """C-ABI sub-matrices of every description in workload ``w``."""
    blocks = w["blocks"]
    out = []
    for bc in w["bcs"]:
        k = bc["kind"]
        if k == "zero":
            out.append(_sub(BC_ZERO, bc["block"], bc["lo"], bc["hi"], bc["comps"]))
        elif k == "const":
            out.append(_sub(BC_CONST, bc["block"], bc["lo"], bc["hi"], bc["comps"],
                            values=np.asarray(bc["values"], np.float64)))
        elif k == "map":
            out.append(_sub(BC_MAP, bc["block"], bc["lo"], bc["hi"], bc["comps"],
                            src_block=bc["src_block"], perm=tuple(bc["perm"]),
                            sign=tuple(bc["sign"]), offset=tuple(bc["offset"])))
        elif k == "interp":
            out.append(_sub(BC_INTERP, bc["block"], bc["lo"], bc["hi"], bc["comps"],
                            p=int(bc["p"]), geometry=BC_GEOM_USER,
                            rot_comp=tuple(bc.get("rot_comp") or (-1, -1)),
                            itp_src_block=np.full(len(bc["axis"]), bc["src_block"], np.int32),
                            itp_start=np.asarray(bc["start"], np.int32).reshape(-1),
                            itp_axis=np.asarray(bc["axis"], np.int32),
                            itp_w=np.asarray(bc["w"], np.float64).reshape(-1),
                            itp_rot=(np.asarray(bc["rot"], np.float64).reshape(-1)
                                     if bc.get("rot_comp") else None)))
        elif k == "csr":
            out.append(_sub(BC_CSR, bc["block"], bc["lo"], bc["hi"], bc["comps"],
                            row_ptr=bc["row_ptr"], col_block=bc["col_block"],
                            col_comp=bc["col_comp"], col_ijk=bc["col_ijk"],
                            val=bc["val"], rhs=bc.get("rhs")))
        elif k == "sync":
            out.append(_sub(BC_SYNC, bc["block"], bc["lo"], bc["hi"], bc["comps"],
                            row_ptr=bc["row_ptr"], col_block=bc["col_block"],
                            col_comp=bc["col_comp"], col_ijk=bc["col_ijk"],
                            val=bc["val"], rhs=bc.get("rhs")))
        elif k == "faces":
            out.extend(faces_submatrices(bc, blocks))
        elif k == "cubed_sphere_edges":
            out.extend(cubed_sphere_submatrices(bc, blocks))
        else:
            raise ValueError(k)
    return out
