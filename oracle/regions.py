"""Region numbering of block-structured variables (Sec. III-A).

Each block owns a data region ``R_D = [0, n0) x [0, n1) x [0, n2)`` and a full
region ``R_F = [-h0, n0 + h0) x ...``; the ghost region is ``R_G = R_F - R_D``.
A block carries ``ncomp`` components (Sec. V-A: several values per grid point)
and ``nlevels`` vertical levels; a sub-matrix row is repeated at every level.

Global numbering used by the oracle (TEST INFRASTRUCTURE ONLY):

* columns of ``A`` -- every data value of every block, block-major, then
  component, level, and the data cell with axis 0 fastest;
* rows of ``A``    -- every full-region value, in the same order as the
  flattened field arrays ``(C, L, F2, F1, F0)`` of all blocks.  Only ghost
  rows are ever populated; the in-place apply leaves data rows as they are.
"""
from __future__ import annotations

import numpy as np


class Layout:
    def __init__(self, blocks):
        self.blocks = blocks
        self.nb = len(blocks)
        self.n = np.array([b["n"] for b in blocks], np.int64).reshape(-1, 3)
        self.h = np.array([b["h"] for b in blocks], np.int64).reshape(-1, 3)
        self.F = self.n + 2 * self.h
        self.L = np.array([b["nlevels"] for b in blocks], np.int64)
        self.C = np.array([b["ncomp"] for b in blocks], np.int64)
        dsz = self.C * self.L * self.n.prod(axis=1)
        fsz = self.C * self.L * self.F.prod(axis=1)
        self.data_base = np.concatenate([[0], np.cumsum(dsz)[:-1]]).astype(np.int64)
        self.full_base = np.concatenate([[0], np.cumsum(fsz)[:-1]]).astype(np.int64)
        self.n_data = int(dsz.sum())
        self.n_full = int(fsz.sum())

    # -- membership --------------------------------------------------------
    def in_data(self, b, ijk):
        ijk = np.asarray(ijk, np.int64).reshape(-1, 3)
        n = self.n[np.asarray(b, np.int64)].reshape(-1, 3)
        return np.all((ijk >= 0) & (ijk < n), axis=1)

    def in_full(self, b, ijk):
        ijk = np.asarray(ijk, np.int64).reshape(-1, 3)
        bb = np.asarray(b, np.int64)
        n, h = self.n[bb].reshape(-1, 3), self.h[bb].reshape(-1, 3)
        return np.all((ijk >= -h) & (ijk < n + h), axis=1)

    # -- numbering -----------------------------------------------------------
    def col(self, b, c, lev, ijk):
        """Column id of data value (block b, comp c, level lev, cell ijk)."""
        b = np.asarray(b, np.int64)
        ijk = np.asarray(ijk, np.int64).reshape(-1, 3)
        n = self.n[b].reshape(-1, 3)
        L = self.L[b]
        cell = (ijk[:, 2] * n[:, 1] + ijk[:, 1]) * n[:, 0] + ijk[:, 0]
        plane = n[:, 0] * n[:, 1] * n[:, 2]
        return self.data_base[b] + (np.asarray(c, np.int64) * L
                                    + np.asarray(lev, np.int64)) * plane + cell

    def row(self, b, c, lev, ijk):
        """Row id of full-region value (block b, comp c, level lev, cell ijk)."""
        b = np.asarray(b, np.int64)
        ijk = np.asarray(ijk, np.int64).reshape(-1, 3)
        F = self.F[b].reshape(-1, 3)
        h = self.h[b].reshape(-1, 3)
        L = self.L[b]
        q = ijk + h
        cell = (q[:, 2] * F[:, 1] + q[:, 1]) * F[:, 0] + q[:, 0]
        plane = F[:, 0] * F[:, 1] * F[:, 2]
        return self.full_base[b] + (np.asarray(c, np.int64) * L
                                    + np.asarray(lev, np.int64)) * plane + cell

    # -- vectors ---------------------------------------------------------------
    def flatten_full(self, fields):
        return np.concatenate([np.asarray(a, np.float64).ravel() for a in fields])

    def unflatten_full(self, y, like):
        out, pos = [], 0
        for a in like:
            out.append(y[pos:pos + a.size].reshape(a.shape))
            pos += a.size
        return out

    def data_vector(self, fields):
        """``x`` over ``R_D`` (FP64) in column order."""
        parts = []
        for blk, a in zip(self.blocks, fields):
            n, h = blk["n"], blk["h"]
            d = np.asarray(a)[:, :, h[2]:h[2] + n[2], h[1]:h[1] + n[1],
                              h[0]:h[0] + n[0]]
            parts.append(np.asarray(d, np.float64).ravel())
        return np.concatenate(parts)

    def data_rows(self):
        """Row ids of every data value (used to scatter ``x_D`` into ``y``)."""
        out = []
        for b, blk in enumerate(self.blocks):
            n = blk["n"]
            k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]),
                                  np.arange(n[0]), indexing="ij")
            ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
            for c in range(blk["ncomp"]):
                for lev in range(blk["nlevels"]):
                    out.append(self.row(np.full(len(ijk), b), c, lev, ijk))
        return np.concatenate(out)


def box_cells(lo, hi):
    """Cells of the box ``[lo, hi)`` with axis 0 fastest, shape (n, 3)."""
    k, j, i = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]),
                          np.arange(lo[0], hi[0]), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.int64)


def ghost_cells(blk):
    """All ghost cells ``R_G`` of a block, in full-array order."""
    n, h = blk["n"], blk["h"]
    cells = box_cells([-h[0], -h[1], -h[2]],
                      [n[0] + h[0], n[1] + h[1], n[2] + h[2]])
    inside = np.all((cells >= 0) & (cells < np.array(n)), axis=1)
    return cells[~inside]
