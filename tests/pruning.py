"""Live ghost values of a stencil (dead-ghost elimination, Sec. IV-C), from
the definition: a ghost cell is live when the stencil, applied at some data
cell, reads it -- the union over offsets o of the data region shifted by o,
minus the data region.  Written with array shifts, independent of the
library's per-cell test."""
import numpy as np


def live_cells(blk, stencil):
    """Boolean (F2, F1, F0) mask of the live ghost cells of one block."""
    n, h = blk["n"], blk["h"]
    F = [n[d] + 2 * h[d] for d in range(3)]
    data = np.zeros((F[2], F[1], F[0]), bool)
    data[h[2]:h[2] + n[2], h[1]:h[1] + n[1], h[0]:h[0] + n[0]] = True
    live = np.zeros_like(data)
    for o in np.asarray(stencil).reshape(-1, 3):
        # live[g] |= data[g - o]
        src = [slice(None)] * 3
        dst = [slice(None)] * 3
        for ax, d in ((2, int(o[0])), (1, int(o[1])), (0, int(o[2]))):
            size = data.shape[ax]
            if abs(d) >= size:
                break
            if d >= 0:
                dst[ax], src[ax] = slice(d, size), slice(0, size - d)
            else:
                dst[ax], src[ax] = slice(0, size + d), slice(-d, size)
        else:
            live[tuple(dst)] |= data[tuple(src)]
    return live & ~data


def live_mask(w, stencil):
    """Flat boolean mask over every value of the workload's fields (the
    order of ``np.concatenate([a.ravel() for a in fields])``)."""
    parts = []
    for a, blk in zip(w["fields"], w["blocks"]):
        m = live_cells(blk, stencil)
        parts.append(np.broadcast_to(m, a.shape).ravel())
    return np.concatenate(parts)
