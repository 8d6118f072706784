"""Host emulation for the exchange tests: the pack layout of bc_pack_run
and the application of a plan's exported rows, in NumPy (test code)."""
import numpy as np

from paper_2605_14780_gb300 import specs


def pack_host(fields, blocks, send):
    """The send buffer bc_pack_run fills: every box of ``send`` (peer,
    block, lo, hi) with all components and levels, [c][l][k][j][i]."""
    parts = []
    for _, b, lo, hi in send:
        h = blocks[b]["h"]
        a = fields[b]
        parts.append(a[:, :, lo[2] + h[2]:hi[2] + h[2], lo[1] + h[1]:hi[1] + h[1],
                       lo[0] + h[0]:hi[0] + h[0]].ravel())
    return np.concatenate(parts) if parts else np.zeros(0, fields[0].dtype)


def staging_views(recvbuf, stage_blocks):
    out, pos = [], 0
    for blk in stage_blocks:
        n = blk["n"]
        shape = (blk["ncomp"], blk["nlevels"], n[2], n[1], n[0])
        cnt = int(np.prod(shape))
        out.append(recvbuf[pos:pos + cnt].reshape(shape))
        pos += cnt
    return out


def apply_rows(ex, arrays, descs):
    """FP64 values of every exported row at every level: a dict
    ``(local slot, element offset) -> value`` (the rows' own sums, in
    entry order)."""
    slots = []
    for a, d in zip(arrays, descs):
        for c in range(d["ncomp"]):
            slots.append((a[c].reshape(-1).astype(np.float64), d["nlevels"],
                          d["level_stride"] if d["nlevels"] > 1 else 0))
    got = {}
    rp = ex["row_ptr"]
    for r in range(len(ex["row_slot"])):
        s = int(ex["row_slot"][r])
        _, L, ls = slots[s]
        for lv in range(L):
            v = ex["rhs"][r]
            for e in range(rp[r], rp[r + 1]):
                cs = int(ex["col_slot"][e])
                xs, _, cls = slots[cs]
                v += ex["val"][e] * xs[int(ex["col_off"][e]) + lv * cls]
            got[(s, int(ex["row_off"][r]) + lv * ls)] = v
    return got


def local_descs(w, part):
    return ([specs.contiguous_block(w["blocks"][b]) for b in part.owned] +
            [specs.contiguous_block(sb) for sb in part.stage_blocks])
