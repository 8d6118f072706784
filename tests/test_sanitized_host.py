"""The plan builder under the address and undefined-behaviour sanitizers:
the host translation units (plan creation, pruning, quadrature rows, the
folding of ghost-reading rows, the work replay) are built with
``-fsanitize=address,undefined`` and a child process builds host-only plans
of every workload type with the sanitizer runtimes preloaded.  Any invalid
access or undefined operation aborts the child.  No GPU."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np
from paper_2605_14780_gb300 import bc, synth
H = {"host_only": 1}
cases = [
    synth.alg1_example(), synth.hpcg_block((5, 4, 3), "P", seed=1),
    synth.hpcg_block((1, 1, 1), "S", seed=1),
    synth.batching(nblocks=10, side_lo=1, side_hi=20, lev_lo=1, lev_hi=7, h=2, seed=3),
    synth.sync_grid(3, 2, 6, 2, 3, 2, "f64", seed=3), synth.two_level(12, 10, 2, 2, 2, "f64", seed=4),
    synth.cubed_sphere(8, 2, 4, 3, ("h", "u", "v"), "f32", seed=5, quad=2),
    synth.cubed_sphere(9, 3, 4, 2, ("h", "u", "v"), "f64", seed=5, quad=3, centred=True, sweeps=4),
    synth.ghost_on_ghost(scheme="smooth", sweeps=5), synth.ghost_on_ghost(scheme="extrapolate"),
    synth.staggered_interp(), synth.swap_xy(synth.staggered_interp(p=6)),
    synth.dirichlet_block(),
]
n = 0
for w in cases:
    for stencil in (None, bc.star_stencil(3 if w["blocks"][0]["n"][2] > 1 else 2, 1)):
        plan = bc.plan_for_workload(w, opts=H, stencil=stencil)
        plan.export_csr()
        checked, bad, msg = plan.check_work()
        assert bad == 0, msg
        n += checked
# rejected descriptions take the error paths
t = synth.tiny_cubed_sphere()
for k in (-1, 65):
    try:
        bc.plan_for_workload(dict(t, ghost_sweeps=k), opts=H)
        raise SystemExit("accepted a bad option")
    except bc.BCError:
        pass
print("values", n)
"""


def _runtime(name):
    gcc = shutil.which("gcc")
    if gcc is None:
        return None
    path = subprocess.run([gcc, f"-print-file-name={name}"], capture_output=True,
                          text=True).stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_plan_builder_is_clean_under_sanitizers():
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan or shutil.which("nvcc") is None:
        pytest.skip("sanitizer runtimes or nvcc not available")
    from paper_2605_14780_gb300.build import build_library
    lib = build_library(sanitize=True)
    env = dict(os.environ, LD_PRELOAD=f"{asan}:{ubsan}", BC_LIBRARY=lib,
               ASAN_OPTIONS="detect_leaks=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1",
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "values" in r.stdout
    assert "runtime error" not in r.stderr, r.stderr[-4000:]
