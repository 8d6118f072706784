"""ctypes binding of the ``libbcgb300`` C ABI (``include/bc.h``).

Argument marshalling only: plans, the forward apply ``y_G = A x_D + b``
(arxiv 2605.14780, Sec. III-B) and its adjoint all run in the library's
sm_103a kernels.  PyTorch supplies device memory and streams.  There is no
fallback: if the compiled library is missing, :func:`load_library` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

LIB_NAME = "libbcgb300.so"
LIB_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib")

BC_F32, BC_F64 = 0, 1
BC_FORM_BATCHED, BC_FORM_TYPEWIDE, BC_FORM_PER_BC = 0, 1, 2
BC_BATCH_PERSISTENT, BC_BATCH_FAMILIES, BC_BATCH_FAMILIES_PERSISTENT, BC_BATCH_SINGLE = 1, 2, 3, 4
STATUS = {0: "BC_OK", 1: "BC_ERR_INVALID_ARG", 2: "BC_ERR_OVERLAP",
          3: "BC_ERR_COLUMN_NOT_DATA", 4: "BC_ERR_UNCOVERED",
          5: "BC_ERR_HALO_TOO_WIDE", 6: "BC_ERR_OUT_OF_RANGE",
          7: "BC_ERR_NOMEM", 8: "BC_ERR_CUDA", 9: "BC_ERR_UNSUPPORTED",
          10: "BC_ERR_TIMEOUT", 11: "BC_ERR_GEOMETRY"}

c_i32, c_i64, c_dbl, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
P_i32 = ctypes.POINTER(c_i32)
P_i64 = ctypes.POINTER(c_i64)
P_dbl = ctypes.POINTER(c_dbl)


class BcBlock(ctypes.Structure):
    _fields_ = [("n", c_i32 * 3), ("h", c_i32 * 3), ("nlevels", c_i32),
                ("ncomp", c_i32), ("stride", c_i64 * 3), ("level_stride", c_i64)]


class BcGrid(ctypes.Structure):
    _fields_ = [("dtype", c_i32), ("nblocks", c_i32),
                ("blocks", ctypes.POINTER(BcBlock))]


class BcSubmatrix(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("block", c_i32), ("lo", c_i32 * 3),
                ("hi", c_i32 * 3), ("ncomps", c_i32), ("comps", P_i32),
                ("values", P_dbl),
                ("src_block", c_i32), ("perm", c_i32 * 3), ("sign", c_i32 * 3),
                ("offset", c_i32 * 3),
                ("p", c_i32), ("geometry", c_i32), ("rot_comp", c_i32 * 2),
                ("cs_panels", c_i32 * 6),
                ("itp_src_block", P_i32), ("itp_start", P_i32),
                ("itp_axis", P_i32), ("itp_w", P_dbl), ("itp_rot", P_dbl),
                ("row_ptr", P_i64), ("col_block", P_i32), ("col_comp", P_i32),
                ("col_ijk", P_i32), ("val", P_dbl), ("rhs", P_dbl),
                ("nquad", c_i32)]


class BcBox(ctypes.Structure):
    _fields_ = [("block", c_i32), ("lo", c_i32 * 3), ("hi", c_i32 * 3)]


class BcPlanOpts(ctypes.Structure):
    _fields_ = [("units_per_lane", c_i32), ("unit_order", c_i32),
                ("threads", c_i32), ("ctas_per_sm", c_i32),
                ("strict_cover", c_i32), ("no_adjoint", c_i32),
                ("no_runs", c_i32), ("host_only", c_i32), ("ghost_sweeps", c_i32),
                ("batch_mode", c_i32), ("scalar_runs", c_i32), ("level_chunk", c_i32),
                ("unstaged_rows", c_i32), ("stencil_fusion", c_i32)]


class BcStats(ctypes.Structure):
    _fields_ = [("ghost_values", c_i64), ("ghost_values_kind", c_i64 * 5),
                ("nitems", c_i64), ("nitems_adjoint", c_i64),
                ("nsubmatrices", c_i64), ("nslots", c_i64),
                ("bytes_fwd", c_i64), ("bytes_adj", c_i64),
                ("table_bytes", c_i64), ("transpose_nnz", c_i64),
                ("element_size", c_i32), ("form_threads", c_i32),
                ("form_ctas_per_sm", c_i32), ("units_per_lane", c_i32),
                ("launches_fwd", c_i32), ("launches_adj", c_i32),
                ("sync_values", c_i64), ("batch_mode", c_i32), ("level_chunk", c_i32)]


#: every function the header declares, with (restype, argtypes)
SIGNATURES = {
    "bc_plan_create": (c_i32, [ctypes.POINTER(BcGrid), ctypes.POINTER(BcSubmatrix),
                               c_i32, ctypes.POINTER(BcPlanOpts),
                               ctypes.POINTER(c_vp)]),
    "bc_plan_create_pruned": (c_i32, [ctypes.POINTER(BcGrid), ctypes.POINTER(BcSubmatrix),
                                      c_i32, ctypes.POINTER(BcPlanOpts),
                                      ctypes.POINTER(c_i32), c_i32,
                                      ctypes.POINTER(c_vp)]),
    "bc_plan_nslots": (c_i32, [c_vp]),
    "bc_apply": (c_i32, [c_vp, c_vp, c_vp]),
    "bc_apply_form": (c_i32, [c_vp, c_vp, c_i32, c_vp]),
    "bc_apply_adjoint": (c_i32, [c_vp, c_vp, c_vp]),
    "bc_apply_host": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "bc_apply_stencil": (c_i32, [c_vp, c_vp, c_vp, P_i32, P_dbl, c_i32, c_vp]),
    "bc_plan_autotune": (c_i32, [c_vp, c_vp, c_vp]),
    "bc_plan_const_values": (c_i32, [c_vp, c_i32, ctypes.POINTER(c_vp), P_i64]),
    "bc_plan_set_const": (c_i32, [c_vp, c_i32, c_vp, c_vp]),
    "bc_plan_check_work": (c_i32, [c_vp, P_i64, P_i64]),
    "bc_plan_stats": (c_i32, [c_vp, ctypes.POINTER(BcStats)]),
    "bc_plan_export_csr": (c_i32, [c_vp, P_i64, P_i64, P_i32, P_i64, P_i64,
                                   P_i32, P_i64, P_dbl, P_dbl]),
    "bc_cubed_sphere_stencils_noalloc": (c_i32, [c_i32, c_i32, c_i32, P_i32, P_i32,
                                                 P_i32, P_dbl, P_dbl]),
    "bc_pack_create": (c_i32, [ctypes.POINTER(BcGrid), ctypes.POINTER(BcBox), c_i32,
                               ctypes.POINTER(c_vp)]),
    "bc_pack_size": (c_i64, [c_vp]),
    "bc_pack_run": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "bc_pack_destroy": (None, [c_vp]),
    "bc_fmap_submatrix": (c_i32, [ctypes.POINTER(BcGrid), c_i32, c_i32, c_i32, c_i32, P_i32,
                                  c_i32, ctypes.POINTER(BcSubmatrix)]),
    "bc_plan_destroy": (None, [c_vp]),
    "bc_status_string": (ctypes.c_char_p, [c_i32]),
    "bc_last_error": (ctypes.c_char_p, []),
}

_LIB = None


def library_path():
    """The in-tree library, or the one ``BC_LIBRARY`` names (e.g. the
    sanitized host build)."""
    return os.environ.get("BC_LIBRARY") or os.path.join(LIB_DIR, LIB_NAME)


def load_library():
    """Load the compiled library (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(
            f"{LIB_NAME} is not built ({path} missing); run "
            "paper_2605_14780_gb300.build.build_library() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class BCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = STATUS.get(status, str(status))


def _check(st):
    if st != 0:
        lib = load_library()
        raise BCError(st, lib.bc_last_error().decode())


def _ptr(arr, ctype):
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


class Plan:
    """A compiled ghost-fill operator.

    ``blocks``: list of dicts ``n, h, nlevels, ncomp, stride, level_stride``
    (element strides); ``subs``: list of sub-matrix dicts as produced by
    :mod:`paper_2605_14780_gb300.specs`; ``dtype``: ``"f32"`` or ``"f64"``;
    ``stencil``: optional ``(n, 3)`` integer offsets of the stencil that
    reads the ghost layers -- the plan then keeps only the ghost values it
    reads (``bc_plan_create_pruned``, dead-ghost elimination).
    """

    def __init__(self, blocks, subs, dtype, opts=None, stencil=None):
        lib = load_library()
        self._lib = lib
        self.dtype = dtype
        self.blocks = blocks
        keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(np.asarray(a, dt))
            keep.append(a)
            return a

        cb = (BcBlock * max(1, len(blocks)))()
        for k, b in enumerate(blocks):
            cb[k].n[:] = list(b["n"])
            cb[k].h[:] = list(b["h"])
            cb[k].nlevels = b["nlevels"]
            cb[k].ncomp = b["ncomp"]
            cb[k].stride[:] = list(b["stride"])
            cb[k].level_stride = b["level_stride"]
        grid = BcGrid(BC_F64 if dtype == "f64" else BC_F32, len(blocks), cb)
        cs = (BcSubmatrix * max(1, len(subs)))()
        for k, s in enumerate(subs):
            m = cs[k]
            m.kind = s["kind"]
            m.block = s["block"]
            m.lo[:] = list(s["lo"])
            m.hi[:] = list(s["hi"])
            comps = arr(s["comps"], np.int32)
            m.ncomps = len(comps)
            m.comps = _ptr(comps, c_i32)
            if s.get("values") is not None:
                m.values = _ptr(arr(s["values"], np.float64), c_dbl)
            m.src_block = s.get("src_block", 0)
            m.perm[:] = list(s.get("perm", (0, 1, 2)))
            m.sign[:] = list(s.get("sign", (1, 1, 1)))
            m.offset[:] = list(s.get("offset", (0, 0, 0)))
            m.p = s.get("p", 0)
            m.geometry = s.get("geometry", 0)
            m.rot_comp[:] = list(s.get("rot_comp", (-1, -1)))
            m.cs_panels[:] = list(s.get("cs_panels", (0, 0, 0, 0, 0, 0)))
            m.nquad = s.get("nquad", 0)
            for key, dt, ct in (("itp_src_block", np.int32, c_i32),
                                ("itp_start", np.int32, c_i32),
                                ("itp_axis", np.int32, c_i32),
                                ("itp_w", np.float64, c_dbl),
                                ("itp_rot", np.float64, c_dbl),
                                ("row_ptr", np.int64, c_i64),
                                ("col_block", np.int32, c_i32),
                                ("col_comp", np.int32, c_i32),
                                ("col_ijk", np.int32, c_i32),
                                ("val", np.float64, c_dbl),
                                ("rhs", np.float64, c_dbl)):
                if s.get(key) is not None:
                    setattr(m, key, _ptr(arr(s[key], dt), ct))
        o = BcPlanOpts()
        for key, v in (opts or {}).items():
            setattr(o, key, v)
        handle = c_vp()
        if stencil is None:
            st = lib.bc_plan_create(ctypes.byref(grid), cs, len(subs),
                                    ctypes.byref(o), ctypes.byref(handle))
        else:
            so = arr(np.asarray(stencil, np.int32).reshape(-1, 3), np.int32)
            st = lib.bc_plan_create_pruned(ctypes.byref(grid), cs, len(subs),
                                           ctypes.byref(o), _ptr(so, c_i32), len(so),
                                           ctypes.byref(handle))
        _check(st)
        self._h = handle
        self.nslots = lib.bc_plan_nslots(handle)
        # the layouts the plan's element offsets were computed for
        self.layout = [dict(b) for b in blocks]

    # -- layout checks -------------------------------------------------------
    def check_tensors(self, tensors):
        """Raise ``ValueError`` unless ``tensors`` (one per block, shaped
        ``(C, L, F2, F1, F0)``) have the dtype and the element strides the
        plan was built for and live on a CUDA device.  The plan's offsets
        are fixed at creation, so a tensor laid out differently would be
        read and written at the wrong elements."""
        want = "torch.float32" if self.dtype == "f32" else "torch.float64"
        if len(tensors) != len(self.layout):
            raise ValueError(f"plan has {len(self.layout)} blocks, got {len(tensors)} tensors")
        for k, (t, b) in enumerate(zip(tensors, self.layout)):
            n, h = b["n"], b["h"]
            shape = (b["ncomp"], b["nlevels"], n[2] + 2 * h[2], n[1] + 2 * h[1],
                     n[0] + 2 * h[0])
            if tuple(t.shape) != shape:
                raise ValueError(f"block {k}: shape {tuple(t.shape)}, plan expects {shape}")
            if str(t.dtype) != want:
                raise ValueError(f"block {k}: dtype {t.dtype}, plan expects {want}")
            # strides matter only along axes with more than one element
            pairs = [(4, b["stride"][0]), (3, b["stride"][1]), (2, b["stride"][2]),
                     (1, b["level_stride"])]
            for dim, s in pairs:
                if shape[dim] > 1 and t.stride(dim) != s:
                    raise ValueError(
                        f"block {k}: stride {t.stride(dim)} along dim {dim}, the plan was "
                        f"built for {s} (strides {tuple(t.stride())})")
            if t.device.type != "cuda":
                raise ValueError(f"block {k}: tensor on {t.device}, the plan runs on CUDA")

    def apply_(self, tensors, form=BC_FORM_BATCHED, stream=None):
        """In-place forward on per-block tensors, after :meth:`check_tensors`."""
        self.check_tensors(tensors)
        self.apply(slot_table(tensors), form, stream)
        return tensors

    def adjoint_(self, tensors, stream=None):
        """In-place adjoint on per-block cotangent tensors laid out as the
        plan's fields, after :meth:`check_tensors`."""
        self.check_tensors(tensors)
        self.adjoint(slot_table(tensors), stream)
        return tensors

    # -- lifecycle -----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.bc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- queries -----------------------------------------------------------
    def stats(self):
        s = BcStats()
        _check(self._lib.bc_plan_stats(self._h, ctypes.byref(s)))
        out = {}
        for name, _ in BcStats._fields_:
            v = getattr(s, name)
            out[name] = list(v) if hasattr(v, "__len__") else int(v)
        return out

    def check_work(self):
        """Host replay of the work lists against the plan's rows:
        ``(values checked, problems, first problem)``."""
        n, bad = c_i64(), c_i64()
        _check(self._lib.bc_plan_check_work(self._h, ctypes.byref(n), ctypes.byref(bad)))
        msg = self._lib.bc_last_error().decode() if bad.value else ""
        return n.value, bad.value, msg

    def export_csr(self):
        nr, nz = c_i64(), c_i64()
        nul = lambda t: ctypes.POINTER(t)()  # noqa: E731
        _check(self._lib.bc_plan_export_csr(
            self._h, ctypes.byref(nr), ctypes.byref(nz), nul(c_i32), nul(c_i64),
            nul(c_i64), nul(c_i32), nul(c_i64), nul(c_dbl), nul(c_dbl)))
        R, E = nr.value, nz.value
        rs = np.zeros(R, np.int32)
        ro = np.zeros(R, np.int64)
        rp = np.zeros(R + 1, np.int64)
        cs = np.zeros(max(E, 1), np.int32)
        co = np.zeros(max(E, 1), np.int64)
        va = np.zeros(max(E, 1), np.float64)
        rh = np.zeros(max(R, 1), np.float64)
        _check(self._lib.bc_plan_export_csr(
            self._h, ctypes.byref(nr), ctypes.byref(nz), _ptr(rs, c_i32),
            _ptr(ro, c_i64), _ptr(rp, c_i64), _ptr(cs, c_i32), _ptr(co, c_i64),
            _ptr(va, c_dbl), _ptr(rh, c_dbl)))
        return {"row_slot": rs, "row_off": ro, "row_ptr": rp,
                "col_slot": cs[:E], "col_off": co[:E], "val": va[:E],
                "rhs": rh[:R]}

    def const_table(self, sub):
        """(device address, length) of the constant table b of BC_CONST
        sub-matrix ``sub``: component-major, box cells axis 0 fastest, in
        the plan's dtype."""
        ptr, n = c_vp(), c_i64()
        _check(self._lib.bc_plan_const_values(self._h, int(sub), ctypes.byref(ptr),
                                              ctypes.byref(n)))
        return ptr.value or 0, n.value

    def const_values(self, sub):
        """The constant table of ``sub`` as a 1-D torch tensor sharing the
        plan's memory (through ``__cuda_array_interface__``), for b = udf(i)
        computed on the device; writes to it change every later apply."""
        import torch
        ptr, n = self.const_table(sub)
        view = _DeviceArray(ptr, n, "<f4" if self.dtype == "f32" else "<f8", owner=self)
        return torch.as_tensor(view, device="cuda")

    def set_const(self, sub, values, stream=None):
        """Copy the device tensor ``values`` (the plan's dtype, the table's
        length, contiguous) into the constant table of ``sub`` on
        ``stream``."""
        _, n = self.const_table(sub)
        want = "torch.float32" if self.dtype == "f32" else "torch.float64"
        if str(values.dtype) != want or values.numel() != n or not values.is_contiguous():
            raise ValueError(f"need a contiguous {want} tensor of {n} values")
        _check(self._lib.bc_plan_set_const(self._h, int(sub), c_vp(values.data_ptr()),
                                           _stream_handle(stream)))

    # -- execution -----------------------------------------------------------
    def apply(self, slot_table, form=BC_FORM_BATCHED, stream=None):
        """Forward apply; ``slot_table`` is a device int64 tensor of slot
        pointers (see :func:`slot_table`)."""
        _check(self._lib.bc_apply_form(self._h, c_vp(slot_table.data_ptr()),
                                       int(form), _stream_handle(stream)))

    def adjoint(self, slot_table, stream=None):
        _check(self._lib.bc_apply_adjoint(self._h, c_vp(slot_table.data_ptr()),
                                          _stream_handle(stream)))

    def apply_stencil(self, slot_table, out_table, offsets, coeffs, stream=None):
        """Ghost fill fused with the stencil ``sum_p coeffs[p] f(x +
        offsets[p])`` (``bc_apply_stencil``): ``out_table`` holds the output
        slots (same layout as the fields); the fields' covered ghosts are
        written as by :meth:`apply`."""
        off = np.ascontiguousarray(np.asarray(offsets, np.int32).reshape(-1, 3))
        cf = np.ascontiguousarray(np.asarray(coeffs, np.float64).reshape(-1))
        if len(cf) != len(off):
            raise ValueError("one weight per stencil point")
        _check(self._lib.bc_apply_stencil(self._h, c_vp(slot_table.data_ptr()),
                                          c_vp(out_table.data_ptr()), _ptr(off, c_i32),
                                          _ptr(cf, c_dbl), len(cf), _stream_handle(stream)))

    def apply_host(self, host_ptrs, dev_ptrs, slot_table, stream=None):
        H = (c_vp * len(host_ptrs))(*host_ptrs)
        D = (c_vp * len(dev_ptrs))(*dev_ptrs)
        _check(self._lib.bc_apply_host(self._h, H, D, c_vp(slot_table.data_ptr()),
                                       _stream_handle(stream)))

    def autotune(self, slot_table, stream=None):
        _check(self._lib.bc_plan_autotune(self._h, c_vp(slot_table.data_ptr()),
                                          _stream_handle(stream)))


def _grid(blocks, dtype):
    cb = (BcBlock * max(1, len(blocks)))()
    for k, b in enumerate(blocks):
        cb[k].n[:] = list(b["n"])
        cb[k].h[:] = list(b["h"])
        cb[k].nlevels = b["nlevels"]
        cb[k].ncomp = b["ncomp"]
        cb[k].stride[:] = list(b["stride"])
        cb[k].level_stride = b["level_stride"]
    return BcGrid(BC_F64 if dtype == "f64" else BC_F32, len(blocks), cb), cb


BC_FMAP_CIRCULAR, BC_FMAP_SYMMETRIC = 0, 1


def fmap_submatrix(blocks, block, axis, side, fmap, comps, dtype="f64"):
    """The C ABI's circular / symmetric face (``bc_fmap_submatrix``) as a
    sub-matrix dict for :class:`Plan`."""
    lib = load_library()
    grid, keep = _grid(blocks, dtype)
    cc = np.ascontiguousarray(np.asarray(comps, np.int32))
    m = BcSubmatrix()
    _check(lib.bc_fmap_submatrix(ctypes.byref(grid), int(block), int(axis), int(side),
                                 int(fmap), _ptr(cc, c_i32), len(cc), ctypes.byref(m)))
    return {"kind": m.kind, "block": m.block, "lo": tuple(m.lo), "hi": tuple(m.hi),
            "comps": [int(c) for c in cc], "src_block": m.src_block, "perm": tuple(m.perm),
            "sign": tuple(m.sign), "offset": tuple(m.offset)}


class Pack:
    """Boxes of blocks packed into one buffer (``bc_pack_create`` /
    ``bc_pack_run``): ``boxes`` is a list of ``(block, lo, hi)``; every
    component and level of a box goes to the buffer, stored
    [component][level][k][j][i], boxes back to back."""

    def __init__(self, blocks, boxes, dtype):
        lib = load_library()
        self._lib = lib
        self._h = None
        grid, keep = _grid(blocks, dtype)
        cbx = (BcBox * max(1, len(boxes)))()
        for k, (b, lo, hi) in enumerate(boxes):
            cbx[k].block = int(b)
            cbx[k].lo[:] = [int(v) for v in lo]
            cbx[k].hi[:] = [int(v) for v in hi]
        handle = c_vp()
        _check(lib.bc_pack_create(ctypes.byref(grid), cbx, len(boxes), ctypes.byref(handle)))
        self._h = handle
        self.size = int(lib.bc_pack_size(handle))

    def run(self, slot_table, buffer, stream=None):
        _check(self._lib.bc_pack_run(self._h, c_vp(slot_table.data_ptr()),
                                     c_vp(buffer.data_ptr()), _stream_handle(stream)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bc_pack_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    """A 1-D device buffer described by ``__cuda_array_interface__`` (keeps
    its plan alive while a view of it exists)."""

    def __init__(self, ptr, n, typestr, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 2,
                                         "strides": None}


def slot_pointers(tensors):
    """Slot pointers of per-block tensors shaped ``(C, L, F2, F1, F0)``: one
    per (block, component), addressing the component's first element."""
    ptrs = []
    for t in tensors:
        for c in range(t.shape[0]):
            ptrs.append(t[c].data_ptr())
    return ptrs


def slot_table(tensors, device=None):
    """Device int64 tensor of :func:`slot_pointers`."""
    import torch
    ptrs = slot_pointers(tensors)
    dev = device or tensors[0].device
    return torch.tensor(ptrs, dtype=torch.int64, device=dev)


def block_descriptors(tensors, blocks):
    """C-ABI block descriptors with the strides of the given tensors."""
    out = []
    for t, b in zip(tensors, blocks):
        out.append({"n": tuple(b["n"]), "h": tuple(b["h"]),
                    "nlevels": b["nlevels"], "ncomp": b["ncomp"],
                    "stride": (t.stride(4), t.stride(3), t.stride(2)),
                    "level_stride": t.stride(1)})
    return out


def plan_for_workload(w, tensors=None, opts=None, stencil=None):
    """Plan of a :mod:`synth` workload (strides of ``tensors`` if given,
    contiguous ``(C, L, F2, F1, F0)`` otherwise), pruned to ``stencil``'s
    reads if given."""
    from . import specs
    if tensors is not None:
        blocks = block_descriptors(tensors, w["blocks"])
    else:
        blocks = [specs.contiguous_block(b) for b in w["blocks"]]
    if w.get("ghost_sweeps"):
        opts = dict(opts or {}, ghost_sweeps=int(w["ghost_sweeps"]))
    return Plan(blocks, specs.submatrices(w), w["dtype"], opts, stencil)


def star_stencil(ndim, radius=1):
    """Offsets of the (2 * ndim * radius + 1)-point star stencil."""
    out = [(0, 0, 0)]
    for d in range(ndim):
        for r in range(1, radius + 1):
            for sgn in (-1, 1):
                o = [0, 0, 0]
                o[d] = sgn * r
                out.append(tuple(o))
    return np.array(out, np.int32)


def box_stencil(ndim, radius=1):
    """Offsets of the (2 * radius + 1)^ndim box stencil."""
    rng = range(-radius, radius + 1)
    z = [0] if ndim < 3 else rng
    return np.array([(i, j, k) for k in z for j in rng for i in rng], np.int32)


class BCFill:
    """``torch.autograd.Function`` of the in-place ghost fill of one plan.

    Forward: ghosts <- A x_D + b in place (the inputs are marked dirty);
    the fields must have the plan's layout (:meth:`Plan.check_tensors`).
    Backward: x_D_bar = y_D_bar + A^T y_G_bar and x_G_bar = 0 on covered
    ghosts, computed in place on copies of the incoming cotangents that are
    laid out with the forward fields' strides, since the plan's element
    offsets were built for those strides.
    """

    _fn = None

    @classmethod
    def function(cls):
        if cls._fn is None:
            import torch

            class _Fill(torch.autograd.Function):
                @staticmethod
                def forward(ctx, plan, *fields):
                    plan.check_tensors(fields)
                    plan.apply(slot_table(fields))
                    ctx.plan = plan
                    ctx.layouts = [(f.size(), f.stride(), f.dtype, f.device) for f in fields]
                    ctx.mark_dirty(*fields)
                    return fields

                @staticmethod
                def backward(ctx, *grads):
                    gs = []
                    for g, (size, stride, dt, dev) in zip(grads, ctx.layouts):
                        out = torch.empty_strided(size, stride, dtype=dt, device=dev)
                        if g is None:
                            out.zero_()
                        else:
                            out.copy_(g)
                        gs.append(out)
                    ctx.plan.adjoint_(gs)
                    return (None, *gs)

            cls._fn = _Fill
        return cls._fn

    @classmethod
    def apply(cls, plan, *fields):
        return cls.function().apply(plan, *fields)


NOALLOC_MAX_CELLS = 65536
NOALLOC_SNAP = 0x100


def cubed_sphere_stencils_noalloc(N, h, p, rotate=True):
    """Cubed-sphere edge stencils from the library's allocation-free entry
    point (for callers that cannot allocate device memory); returns host
    arrays ``nb, node0 (n, 2), axis, w (n, p), rot (n, 2, 2) | None`` in the
    order panel, strip (axis-0 low/high, axis-1 low/high), depth, along."""
    lib = load_library()
    n = 24 * N * h
    nb = np.zeros(n, np.int32)
    node0 = np.zeros((n, 2), np.int32)
    axis = np.zeros(n, np.int32)
    w = np.zeros((n, p), np.float64)
    rot = np.zeros((n, 2, 2), np.float64) if rotate else None
    _check(lib.bc_cubed_sphere_stencils_noalloc(
        int(N), int(h), int(p), _ptr(nb, c_i32), _ptr(node0, c_i32),
        _ptr(axis, c_i32), _ptr(w, c_dbl),
        _ptr(rot, c_dbl) if rotate else ctypes.POINTER(c_dbl)()))
    return {"nb": nb, "node0": node0, "axis": axis, "w": w, "rot": rot}
