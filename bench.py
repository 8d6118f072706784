"""Throughput of the ghost-fill operator y_G = A x_D + b on one GB300 per rank.

Headline workload: 512 uneven 2-D blocks (sides log-uniform in [16, 256],
1-64 levels, h = 2, FP32), every edge drawing a halo copy, circular or
symmetric map, zero padding or a CSR user matrix, corners zero.  The plan is
autotuned first (bc_plan_autotune; --no-autotune keeps its defaults); one
step is one batched, graph-captured apply of the whole operator.  The JSON
line also carries the per-sub-matrix and per-kind launch forms, the
end-to-end number from host memory, the roofline of the dominant kernel, the
FP64 oracle's product on the host cores, the other workloads of the scope
table (with their sector-granular DRAM floors), the fused boundary-and-
stencil workload, and the SM clocks seen during the timed loop.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --oracle-all     # the oracle on every workload, then exit
    python bench.py --profile-case batching:level_innermost:struct   # for ncu

Multi-GPU runs are independent replicas (the operator has no exchange step
on one GPU's resident blocks): value = all ranks' ghost values / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("ghost cells/s and HBM GB/s (% of 8 TB/s), batched vs per-BC "
          "launches, 1 GB300")
UNIT = "ghost values/s"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 8000.0
FP64_TFLOPS = 1.25  # non-tensor FP64 of the part (nominal)


# ----------------------------------------------------------------------------
# distributed helpers (replicas only)
# ----------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value, world, device=None):
    """Max of a float over ranks (identity for one rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(values_per_rank, times_per_rank):
    """Whole-job throughput of independent replicas: sum of the units every
    rank processed divided by the slowest rank's time."""
    return float(sum(values_per_rank)) / float(max(times_per_rank))


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        # the samples file: BC_CLOCKS_DIR if set, else the system temp dir
        out = os.environ.get("BC_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"bc_clocks_rank{device_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
                power.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        load = [s for s, pw in zip(sm, power) if pw > 0.25 * max(power)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kernels.cu", "bc_internal.h"):
        with open(os.path.join(ROOT, "paper_2605_14780_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[workload]
        if e.get("kernel_source") != kernel_source_hash():
            return None
        return {"dram_bytes_per_launch": int(e["dram_bytes_per_launch"]),
                "l2_write_bytes": int(e.get("l2_write_bytes", 0)) or None}
    except Exception:
        return None


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
def make_workload(name):
    from paper_2605_14780_gb300 import synth
    if name == "batching":
        return synth.batching(), ("batching: 512 2-D blocks, sides log-uniform "
                                  "in [16, 256], 1-64 levels, h=2, FP32, "
                                  "per-edge halo/circular/symmetric/zero/CSR, "
                                  "corners zero")
    if name == "swe":
        return synth.swe_cubed_sphere(), ("cubed sphere 6 x 384^2, h=3, "
                                          "(h,u,v) x 32 levels FP32, p=6")
    if name == "adjoint":
        return synth.adjoint_cubed_sphere(), ("cubed sphere 6 x 768^2, h=3, "
                                              "(h,u,v) x 32 levels FP32, p=6")
    if name == "sync":
        return (synth.sync_grid(8, 8, 129, 3, 32, 3, "f32", seed=12),
                "block-edge averaging: 8 x 8 node-centred blocks of 129^2 nodes "
                "sharing their edges, h=3, 3 components x 32 levels FP32")
    if name == "hope":
        return synth.hope_cubed_sphere(), ("cubed sphere 6 x 384^2, h=3, (h,u,v) x 32 "
                                           "levels FP32, cell averages by 4x4 reconstruction "
                                           "at 2x2 Gauss points (CSR rows of 16/32 entries)")
    if name == "hpcg":
        return synth.hpcg_block(128, "P"), "HPCG-like 128^3 FP64, h=1, x periodic"
    raise ValueError(name)


def make_workload_named(name):
    from paper_2605_14780_gb300 import synth
    if name == "tiny":
        return synth.tiny_cubed_sphere()
    return make_workload(name)[0]


def field_copies(w, ncopies, device, layout="level_outermost"):
    """``ncopies`` independent device copies of the fields, each copy one
    contiguous allocation with the blocks back to back.  ``layout``:
    ``level_outermost`` stores each component as [level][k][j][i];
    ``level_innermost`` as [k][j][i][level] (views keep the (C, L, F2, F1,
    F0) index order, the plan reads the strides)."""
    import torch
    sizes = [a.size for a in w["fields"]]
    dt = torch.float32 if w["dtype"] == "f32" else torch.float64
    copies = []
    for _ in range(ncopies):
        buf = torch.empty(sum(sizes), dtype=dt, device=device)
        views = layout_views(buf, w, layout)
        for v, a in zip(views, w["fields"]):
            v.copy_(torch.from_numpy(a))
        copies.append((buf, views))
    return copies


def layout_views(buf, w, layout):
    """Per-block (C, L, F2, F1, F0) views of one flat buffer in ``layout``."""
    views, pos = [], 0
    for a in w["fields"]:
        if layout == "level_innermost":
            C, L, F2, F1, F0 = a.shape
            v = buf[pos:pos + a.size].view(C, F2, F1, F0, L).permute(0, 4, 1, 2, 3)
        else:
            v = buf[pos:pos + a.size].view(a.shape)
        views.append(v)
        pos += a.size
    return views


def measure_forward(w, device, stream, steps, warmup, layout="level_outermost",
                    adjoint=False, floor=False, stencil=None, autotune=True):
    """Device time of the batched forward (and optionally the adjoint) of a
    workload with rotating field copies, after bc_plan_autotune; returns a
    dict of numbers."""
    from paper_2605_14780_gb300 import bc
    esize = 4 if w["dtype"] == "f32" else 8
    field_bytes = sum(a.size for a in w["fields"]) * esize
    ncopies = int(min(8, max(2, np.ceil(3 * 256e6 / field_bytes) + 1)))
    copies = field_copies(w, ncopies, device, layout)
    plan = bc.plan_for_workload(w, copies[0][1], stencil=stencil)
    tables = [bc.slot_table(v) for _, v in copies]
    if autotune:
        plan.autotune(tables[0])
    st = plan.stats()
    hbm, _ = measured_peaks()
    gs = [capture(lambda t=t: plan.apply(t, stream=stream), stream) for t in tables]
    per, tot = time_steps([g.replay for g in gs], steps, warmup, stream, 1)
    ms = tot / steps
    out = {"ghost_values": int(st["ghost_values"]), "ms": ms,
           "ghost_values_per_s": st["ghost_values"] / (ms / 1e3),
           "algorithmic_bytes": int(st["bytes_fwd"]),
           "useful_gbs": st["bytes_fwd"] / (ms / 1e3) / 1e9,
           "frac_of_measured_hbm": st["bytes_fwd"] / (ms / 1e3) / 1e9 / hbm,
           "layout": layout, "field_copies": ncopies,
           "form": FORM_DESC.get(st["batch_mode"], str(st["batch_mode"])),
           "threads": st["form_threads"], "units_per_lane": st["units_per_lane"],
           "level_chunk": st["level_chunk"]}
    if floor:
        out["dram_floor"] = dram_floor(plan, w, copies[0][1], copies[0][0])
        for g in (32, 64):
            fb = out["dram_floor"][f"granule_{g}B_bytes"]
            out["dram_floor"][f"frac_of_floor_{g}B"] = fb / (ms / 1e3) / 1e9 / hbm
    del gs
    if adjoint:
        ga = [capture(lambda t=t: plan.adjoint(t, stream=stream), stream) for t in tables]
        per, tot = time_steps([g.replay for g in ga], steps, warmup, stream, 1)
        ams = tot / steps
        out["adjoint"] = {"ms": ams, "ghost_values_per_s": st["ghost_values"] / (ams / 1e3),
                          "algorithmic_bytes": int(st["bytes_adj"]),
                          "useful_gbs": st["bytes_adj"] / (ams / 1e3) / 1e9,
                          "frac_of_measured_hbm": st["bytes_adj"] / (ams / 1e3) / 1e9 / hbm,
                          "launches_per_step": 2}
        del ga
    del copies, tables, plan
    import torch
    torch.cuda.empty_cache()
    return out


def measure_fused(device, stream, steps, warmup, nblocks=16):
    """The ghost fill fused with the 27-point operator (diagonal 26,
    off-diagonals -1) on ``nblocks`` independent 128^3 FP64 blocks, x
    periodic and zero elsewhere: one bc_apply_stencil per step.  FP64 on
    this GPU: 27 fused multiply-adds per output make it bound by the FP64
    pipes, not by HBM."""
    from paper_2605_14780_gb300 import bc, synth
    w = synth.hpcg_block(128, "P", seed=2, nblocks=nblocks)
    offs = bc.box_stencil(3, 1)
    cf = np.array([26.0 if tuple(o) == (0, 0, 0) else -1.0 for o in offs])
    copies = field_copies(w, 2, device)
    outs = field_copies(w, 2, device)
    plan = bc.plan_for_workload(w, copies[0][1], {"stencil_fusion": 1})
    tabs = [bc.slot_table(v) for _, v in copies]
    otabs = [bc.slot_table(v) for _, v in outs]
    gs = [capture(lambda k=k: plan.apply_stencil(tabs[k], otabs[k], offs, cf, stream=stream),
                  stream) for k in range(2)]
    per, tot = time_steps([g.replay for g in gs], steps, warmup, stream, 1)
    ms = tot / steps
    nd = nblocks * 128 ** 3
    ng = nblocks * (130 ** 3 - 128 ** 3)
    byts = (nd + ng) * 8 + (nd + ng) * 8   # read every value, write outputs and ghosts
    flops = 2 * len(cf) * nd
    st = plan.stats()
    return {"workload": f"{nblocks} x 128^3 FP64 blocks, x periodic, 27-point operator",
            "ms": ms, "outputs": nd, "ghost_values": int(st["ghost_values"]),
            "outputs_per_s": nd / (ms / 1e3),
            "useful_gbs": byts / (ms / 1e3) / 1e9,
            "frac_of_measured_hbm": byts / (ms / 1e3) / 1e9 / measured_peaks()[0],
            "fp64_tflops": flops / (ms / 1e3) / 1e12,
            "roofline": {"bound": "alu", "achieved": flops / (ms / 1e3) / 1e12,
                         "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                         "frac": flops / (ms / 1e3) / 1e12 / FP64_TFLOPS,
                         "peak_source": "nominal FP64 rate of the part (no measured FP64 peak)"}}


def capture(fn, stream):
    import torch
    with torch.cuda.stream(stream):
        fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fn()
    return g


def time_steps(step_fns, steps, warmup, stream, world, min_warm_s=0.0):
    """Run ``warmup`` untimed and exactly ``steps`` timed steps (step i uses
    ``step_fns[i % len]``), each bracketed by CUDA events on ``stream``;
    returns per-step device times (ms) and the total (ms)."""
    import torch
    with torch.cuda.stream(stream):
        t0 = time.time()
        i = 0
        while i < warmup or time.time() - t0 < min_warm_s:
            step_fns[i % len(step_fns)]()
            i += 1
            if i % 64 == 0:
                stream.synchronize()
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for s in range(steps):
            step_fns[s % len(step_fns)]()
            ev[s + 1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
    per = [ev[s].elapsed_time(ev[s + 1]) for s in range(steps)]
    return per, ev[0].elapsed_time(ev[steps])


# ----------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline / reference arm)
# ----------------------------------------------------------------------------
def oracle_timing(w, budget_s=12.0, max_reps=None):
    """The FP64 oracle's product ``g = A x + b`` on the host cores, timed
    alone: ``A`` (explicit CSR) and ``x`` (the data values in FP64) are built
    first, outside the timing.  SciPy's CSR product runs on one core."""
    from oracle.operator import build_operator
    t0 = time.time()
    op = build_operator(w)
    x = op.layout.data_vector(w["fields"])
    t_build = time.time() - t0
    reps, t_apply = 0, 0.0
    while t_apply < budget_s and (max_reps is None or reps < max_reps):
        t1 = time.time()
        g = op.A @ x + op.b
        t_apply += time.time() - t1
        reps += 1
    del g
    nvals = len(op.rows)
    return {"value": nvals * reps / t_apply, "unit": UNIT, "cores": 1,
            "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"full workload ({nvals} ghost values): {reps} FP64 SciPy CSR "
                       f"products g = A x + b in {t_apply:.1f} s on one core (of "
                       f"{os.cpu_count()}), after {t_build:.1f} s building A and x"),
            "spmv_s": t_apply / reps, "build_s": t_build}


def run_reference(args, rank, world):
    if rank != 0:
        return
    w, desc = make_workload(args.workload)
    from oracle.operator import build_operator
    t0 = time.time()
    op = build_operator(w)
    x = op.layout.data_vector(w["fields"])
    t_build = time.time() - t0
    for _ in range(args.warmup):
        op.A @ x + op.b
    times = []
    for _ in range(args.steps):
        t1 = time.time()
        op.A @ x + op.b
        times.append(time.time() - t1)
    nvals = len(op.rows)
    value = nvals * len(times) / sum(times)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": desc, "ghost_values": nvals},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1,
                         "host_cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"full workload, {len(times)} timed FP64 SciPy CSR "
                                   f"products g = A x + b on one core after "
                                   f"{t_build:.1f} s building A and x"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def oracle_all(args):
    """The oracle's product timed on every workload of the scope table
    (``--oracle-all``; several minutes)."""
    out = {}
    for name in ("tiny", "hpcg", "swe", "batching", "adjoint"):
        w = make_workload_named(name)
        out[name] = oracle_timing(w, budget_s=args.oracle_budget_s)
        del w
        print(json.dumps({name: out[name]}), flush=True)
    return out


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def dram_floor(plan, w, views, buf):
    """Smallest DRAM traffic one forward apply can cause: every 32- or 64-byte
    granule it reads, every granule it writes, and one extra read for each
    granule it writes only partly (HBM3e with ECC has no write mask).  Built
    from the plan's own rows (bc_plan_export_csr) and the fields' addresses."""
    ex = plan.export_csr()
    esize = buf.element_size()
    base = buf.data_ptr()
    slot_addr, slot_ls, slot_L = [], [], []
    for v, blk in zip(views, w["blocks"]):
        for c in range(blk["ncomp"]):
            slot_addr.append((v[c].data_ptr() - base) // esize)
            slot_ls.append(v.stride(1))
            slot_L.append(blk["nlevels"])
    slot_addr = np.array(slot_addr, np.int64)
    slot_ls = np.array(slot_ls, np.int64)
    slot_L = np.array(slot_L, np.int64)

    def expand(slots, offs):
        L = slot_L[slots]
        rep = np.repeat(np.arange(len(slots)), L)
        lev = np.arange(L.sum()) - np.repeat(np.cumsum(L) - L, L)
        return slot_addr[slots][rep] + offs[rep] + lev * slot_ls[slots][rep]

    wr = expand(ex["row_slot"], ex["row_off"])
    rd = expand(ex["col_slot"], ex["col_off"])
    out = {"source_values": int(len(np.unique(rd)))}
    for g in (32, 64):
        per = g // esize
        wsec, wcnt = np.unique(wr // per, return_counts=True)
        partial = wsec[wcnt < per]
        rsec = np.union1d(np.unique(rd // per), partial)
        out[f"granule_{g}B_bytes"] = int((len(wsec) + len(rsec)) * g)
    return out


FAMILY_KINDS = {"structured (zero/const/map)": (0, 1, 2), "interpolation": (3,),
                "csr": (4,)}


def family_plans(w, tensors, opts=None):
    """One plan per kernel family over the same fields (with the options
    ``opts``), to time each family's kernel on its own."""
    from paper_2605_14780_gb300 import bc, specs
    subs = specs.submatrices(w)
    blocks = bc.block_descriptors(tensors, w["blocks"])
    base = dict(opts or {}, no_adjoint=1, batch_mode=bc.BC_BATCH_FAMILIES)
    out = {}

    def family_kind(s):
        # reconstruction-and-quadrature rows are executed as user CSR rows
        if s["kind"] == specs.BC_INTERP and s.get("geometry") in (
                specs.BC_GEOM_CUBED_SPHERE_QUAD, specs.BC_GEOM_CUBED_SPHERE_QUAD_CENTRED):
            return specs.BC_CSR
        return s["kind"]
    for name, kinds in FAMILY_KINDS.items():
        part = [s for s in subs if family_kind(s) in kinds]
        if part:
            out[name] = bc.Plan(blocks, part, w["dtype"], base)
    return out


def run_ours(args, rank, world, local):
    import torch
    from paper_2605_14780_gb300 import bc

    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    w, desc = make_workload(args.workload)
    esize = 4 if w["dtype"] == "f32" else 8
    field_bytes = sum(a.size for a in w["fields"]) * esize
    ncopies = max(2, int(np.ceil(3 * 256e6 / field_bytes)) + 1)
    ncopies = min(ncopies, 8)
    copies = field_copies(w, ncopies, device, args.layout)
    plan = bc.plan_for_workload(w, copies[0][1])
    tables = [bc.slot_table(v) for _, v in copies]
    tune_s = None
    if not args.no_autotune:
        t0 = time.time()
        plan.autotune(tables[0])
        tune_s = time.time() - t0
    st = plan.stats()
    nvals = st["ghost_values"]
    stream = torch.cuda.Stream(device)
    hbm, peak_kind = measured_peaks()

    def graphs_for(pl, form=bc.BC_FORM_BATCHED):
        return [capture(lambda t=t: pl.apply(t, form, stream=stream), stream)
                for t in tables]

    # -- headline: batched form (one fork/join group of family kernels) -----
    g_batched = graphs_for(plan)
    sampler = ClockSampler(local)
    sampler.start()
    per, total = time_steps([g.replay for g in g_batched], args.steps,
                            args.warmup, stream, world,
                            min_warm_s=args.min_warm_s)
    clocks = sampler.stop()
    del g_batched
    t_step = total / args.steps
    t_max = reduce_max(total, world, device)
    value = nvals * args.steps * world / (t_max / 1e3)
    step_gbs = st["bytes_fwd"] / (statistics.mean(per) / 1e3) / 1e9

    # -- each family kernel on its own: the roofline of the dominant one ----
    kernels = {}
    if not args.only_batched:
        tuned = {"threads": st["form_threads"], "units_per_lane": st["units_per_lane"],
                 "level_chunk": st["level_chunk"]}
        for name, fp in family_plans(w, copies[0][1], tuned).items():
            fst = fp.stats()
            gs = graphs_for(fp)
            pk, tk = time_steps([g.replay for g in gs], min(args.steps, 500), 5,
                                stream, world)
            ms = statistics.mean(pk)
            kernels[name] = {"ms": ms, "algorithmic_bytes": int(fst["bytes_fwd"]),
                             "ghost_values": int(fst["ghost_values"]),
                             "achieved_gbs": fst["bytes_fwd"] / (ms / 1e3) / 1e9}
            kernels[name]["frac"] = kernels[name]["achieved_gbs"] / hbm
            del gs, fp
    if kernels:
        dom_name = max(kernels, key=lambda k: kernels[k]["ms"])
        dom = kernels[dom_name]
    else:
        dom_name, dom = "batched step", {"ms": statistics.mean(per),
                                         "algorithmic_bytes": st["bytes_fwd"],
                                         "achieved_gbs": step_gbs}

    # -- baselines: per-kind and per-sub-matrix launches ---------------------
    forms = {"batched": {"ms": t_step, "launches_per_step": "1 graph: one kernel per family, concurrent"}}
    for name, form, nsteps in [] if args.only_batched else (("typewide", bc.BC_FORM_TYPEWIDE, min(args.steps, 200)),
                               ("per_bc", bc.BC_FORM_PER_BC, min(args.steps, 20))):
        gs = graphs_for(plan, form)
        p2, tot2 = time_steps([g.replay for g in gs], nsteps, 3, stream, world)
        nl = 5 if form == bc.BC_FORM_TYPEWIDE else st["nsubmatrices"]
        forms[name] = {"ms": tot2 / nsteps, "launches_per_step": int(nl),
                       "ghost_values_per_s": nvals / (tot2 / nsteps / 1e3)}
        del gs
    if not args.only_batched:
        forms["speedup_batched_vs_per_bc"] = forms["per_bc"]["ms"] / t_step
        forms["speedup_batched_vs_typewide"] = forms["typewide"]["ms"] / t_step

    # -- end to end from host memory -----------------------------------------
    # (a) the fields stay in pinned host memory and the plan's kernels read
    #     their sources and write the ghosts through the host link (slot
    #     pointers of mapped host memory; nothing is staged on the device);
    # (b) bc_apply_host: whole slots copied to the device, applied, copied
    #     back.
    e2e = None
    if not args.only_batched:
        host = torch.empty(copies[0][0].numel(), dtype=copies[0][0].dtype).pin_memory()
        host.copy_(copies[0][0].cpu())
        hviews = layout_views(host, w, args.layout)
        hptrs = bc.slot_pointers(hviews)
        htable = torch.tensor(hptrs, dtype=torch.int64, device=device)
        e2e_steps = max(3, min(args.steps, 50))
        pz, totz = time_steps([lambda: plan.apply(htable, stream=stream)], e2e_steps, 3,
                              stream, world)
        z_ms = reduce_max(totz, world, device) / e2e_steps
        dptrs = bc.slot_pointers(copies[0][1])
        c_steps = max(3, min(args.steps, 20))
        pe, tote = time_steps(
            [lambda: plan.apply_host(hptrs, dptrs, tables[0], stream=stream)],
            c_steps, 2, stream, world)
        e2e_ms = reduce_max(tote, world, device) / c_steps
        src_values = dram_floor(plan, w, copies[0][1], copies[0][0])["source_values"]
        e2e = {"value": nvals * world / (z_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(src_values * esize),
               "d2h_bytes_per_step": int(nvals * esize), "ms_per_step": z_ms,
               "path": ("fields in pinned host memory: one bc_apply whose kernels read "
                        "the sources and write the ghost values through the host link "
                        "(h2d = the distinct source values read, d2h = the ghost values "
                        "written)"),
               "copies": {"value": nvals * world / (e2e_ms / 1e3), "ms_per_step": e2e_ms,
                          "h2d_bytes_per_step": int(field_bytes),
                          "d2h_bytes_per_step": int(field_bytes),
                          "path": "bc_apply_host: every slot copied in, applied, copied out"}}

    traffic = profiled_traffic(f"{args.workload}:{args.layout}:{dom_name}")
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": w["dtype"], "data": "synthetic",
        "config": {"workload": desc, "ghost_values": int(nvals),
                   "layout": LAYOUT_DESC[args.layout],
                   "form": FORM_DESC.get(st["batch_mode"], str(st["batch_mode"])),
                   "threads": st["form_threads"],
                   "autotuned": tune_s is not None,
                   "autotune_s": tune_s,
                   "level_chunk": st["level_chunk"],
                   "units_per_lane": st["units_per_lane"],
                   "l2": (f"{ncopies} rotating copies of the fields "
                          f"({ncopies * field_bytes / 1e9:.2f} GB), a copy is "
                          f"reused every {ncopies} steps"),
                   "parallelism": f"replicas x{world}"},
        "hbm_gbs_useful": step_gbs,
        "pct_of_8tbs": 100.0 * step_gbs / NOMINAL_HBM_GBS,
        "roofline": {"bound": "hbm", "kernel": dom_name,
                     "achieved": dom["achieved_gbs"], "peak": hbm,
                     "unit": "GB/s", "frac": dom["achieved_gbs"] / hbm,
                     "peak_source": peak_kind,
                     "traffic": (traffic or {}).get("dram_bytes_per_launch"),
                     "traffic_note": ("DRAM read + write bytes of one launch (ncu); the "
                                      "stores stay in L2 during a short replay, so "
                                      "l2_write_bytes (L2 write sectors x 32) counts them"),
                     "l2_write_bytes": (traffic or {}).get("l2_write_bytes"),
                     "algorithmic_bytes_per_launch": int(dom["algorithmic_bytes"]),
                     "kernel_ms": dom["ms"],
                     "step": {"algorithmic_bytes": int(st["bytes_fwd"]),
                              "achieved": step_gbs, "frac": step_gbs / hbm}},
        "kernels": kernels,
        "forms": forms,
        "e2e": e2e,
        "gpu_launches": args.steps * n_family_kernels(st),
        "clocks": clocks,
    }
    if not args.only_batched:
        result["dram_floor"] = dram_floor(plan, w, copies[0][1], copies[0][0])
    if not args.only_batched and not args.no_variants:
        other = "level_outermost" if args.layout == "level_innermost" else "level_innermost"
        result["layout_variants"] = {other: measure_forward(
            w, device, stream, min(args.steps, 500), 5, other, floor=True,
            autotune=not args.no_autotune)}
        # the other workloads of the scope table, batched forward (+ adjoint)
        others = {}
        for name, fn, adj in (
                ("tiny_cubed_sphere_6x32", lambda: make_workload_named("tiny"), False),
                ("hpcg_128_P", lambda: make_workload_named("hpcg"), False),
                ("swe_cubed_sphere_6x384_L32", lambda: make_workload_named("swe"), False),
                ("adjoint_cubed_sphere_6x768_L32", lambda: make_workload_named("adjoint"), True),
                ("sync_grid_8x8_n129_L32", lambda: make_workload_named("sync"), True)):
            ww = fn()
            others[name] = measure_forward(ww, device, stream, min(args.steps, 300), 5,
                                           adjoint=adj, floor=True,
                                           autotune=not args.no_autotune)
            del ww
        # reconstruction-and-quadrature rows (user CSR rows of 16 / 32
        # entries); recorded as an error entry rather than losing the line
        # if this newer path fails
        try:
            ww = make_workload_named("hope")
            others["hope_cubed_sphere_6x384_L32_p4_q2"] = measure_forward(
                ww, device, stream, min(args.steps, 300), 5, adjoint=True, floor=True,
                autotune=not args.no_autotune)
            del ww
        except Exception as e:  # noqa: BLE001
            others["hope_cubed_sphere_6x384_L32_p4_q2"] = {"error": f"{type(e).__name__}: {e}"}
        # boundary rows fused with the stencil that reads them (Sec. IV-C)
        try:
            others["fused_27pt_hpcg_16x128"] = measure_fused(device, stream,
                                                             min(args.steps, 50), 3)
        except Exception as e:  # noqa: BLE001
            others["fused_27pt_hpcg_16x128"] = {"error": f"{type(e).__name__}: {e}"}
        result["other_workloads"] = others
        # dead-ghost elimination (Sec. IV-C): the same workloads, plans cut
        # to the ghost values a following stencil reads
        pruned = {}
        for name, fn, lay, stc in (
                ("batching_star5_levels_innermost", lambda: w, "level_innermost",
                 bc.star_stencil(2, 1)),
                ("batching_box9_levels_innermost", lambda: w, "level_innermost",
                 bc.box_stencil(2, 1)),
                ("hpcg_128_P_7pt", lambda: make_workload_named("hpcg"), "level_outermost",
                 bc.star_stencil(3, 1))):
            ww = fn()
            pruned[name] = measure_forward(ww, device, stream, min(args.steps, 300), 5, lay,
                                           stencil=stc)
            pruned[name]["stencil_points"] = int(len(stc))
            del ww
        result["pruned_variants"] = pruned
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = oracle_timing(w)
    if rank == 0:
        print(json.dumps(result))


def n_family_kernels(st):
    """Kernels of one batched apply, as the plan counts them (one per
    non-empty kernel family, the run records, Sync rows)."""
    return int(st["launches_fwd"])


def profile_case(spec):
    """A few applies of one case, for a profiler capture of one launch:
    ``<workload>:<layout>:<what>`` with what = struct | interp | csr (that
    family's plan alone), all (the batched apply), adjoint, or fused (the
    27-point fused workload on 4 blocks)."""
    import torch
    from paper_2605_14780_gb300 import bc, synth
    wname, layout, what = spec.split(":")
    dev = torch.device("cuda", 0)
    if what == "fused":
        w = synth.hpcg_block(128, "P", seed=2, nblocks=4)
        offs = bc.box_stencil(3, 1)
        cf = np.array([26.0 if tuple(o) == (0, 0, 0) else -1.0 for o in offs])
        copies = field_copies(w, 2, dev)
        outs = field_copies(w, 2, dev)
        plan = bc.plan_for_workload(w, copies[0][1], {"stencil_fusion": 1})
        for k in range(4):
            plan.apply_stencil(bc.slot_table(copies[k % 2][1]), bc.slot_table(outs[k % 2][1]),
                               offs, cf)
    else:
        w = make_workload_named(wname)
        copies = field_copies(w, 2, dev, layout)
        tables = [bc.slot_table(v) for _, v in copies]
        if what in ("all", "adjoint"):
            plan = bc.plan_for_workload(w, copies[0][1])
        else:
            name = {"struct": "structured (zero/const/map)", "csr": "csr",
                    "interp": "interpolation"}[what]
            plan = family_plans(w, copies[0][1])[name]
        for k in range(4):
            (plan.adjoint if what == "adjoint" else plan.apply)(tables[k % 2])
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": spec, "bytes_fwd": plan.stats()["bytes_fwd"],
                      "bytes_adj": plan.stats()["bytes_adj"]}))


FORM_DESC = {
    1: "batched, persistent: one resident grid claiming the items of every kind",
    2: "batched: one graph launch, one plain-grid kernel per family, concurrent",
    3: "batched: one persistent kernel per family, concurrent",
    4: "batched: one plain-grid kernel over every item of every kind, longest first",
}

LAYOUT_DESC = {
    "level_innermost": "levels innermost: each component stored [k][j][i][level]",
    "level_outermost": "levels outermost: each component stored [level][k][j][i]",
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batching",
                    choices=["batching", "swe", "adjoint", "hpcg", "sync", "hope"])
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the plan's default options (no bc_plan_autotune)")
    ap.add_argument("--oracle-all", action="store_true",
                    help="time the oracle's product on every workload and exit")
    ap.add_argument("--oracle-budget-s", type=float, default=10.0)
    ap.add_argument("--profile-case", default=None,
                    help="<workload>:<layout>:<struct|interp|csr|all|adjoint|fused>: a few "
                         "applies of one case for a profiler capture, then exit")
    ap.add_argument("--layout", default="level_innermost",
                    choices=["level_innermost", "level_outermost"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the layout variant and the other workloads")
    ap.add_argument("--only-batched", action="store_true",
                    help="time the batched form only (for profiler runs)")
    ap.add_argument("--min-warm-s", type=float, default=1.0,
                    help="minimum seconds of warm-up before the timed steps")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.oracle_all:
        if rank == 0:
            print(json.dumps({"oracle_all": oracle_all(args)}))
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
