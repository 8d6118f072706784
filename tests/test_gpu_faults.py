"""Failure paths made on the host: BC_FAULT_INJECT=alloc:<n> makes the n-th
device allocation of a plan creation fail (no GPU fault is made).  Creation
must report BC_ERR_NOMEM, leak no device memory, and leave the library
usable."""
import pytest

from gpu_util import compare, to_device
from paper_2605_14780_gb300 import bc, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make,counts", [
    (lambda: synth.batching(nblocks=20, side_lo=3, side_hi=24, lev_lo=1, lev_hi=6, h=2,
                            seed=31, dtype="f32"), (1, 2)),
    (lambda: synth.cubed_sphere(8, 2, 4, 2, ("h", "u", "v"), "f64", seed=32), (1, 3, 5, 6, 7)),
])
def test_allocation_failures_report_nomem_without_leaks(monkeypatch, make, counts):
    import torch
    w = make()
    ts = to_device(w["fields"])
    # one good plan first: the library's kernels (and their static device
    # arrays) load lazily on first use, which is not a leak
    bc.plan_for_workload(w, ts).apply(bc.slot_table(ts))
    torch.cuda.synchronize()
    ts = to_device(w["fields"])
    free0 = torch.cuda.mem_get_info()[0]
    for n in counts:
        monkeypatch.setenv("BC_FAULT_INJECT", f"alloc:{n}")
        for _ in range(5):
            with pytest.raises(bc.BCError) as e:
                bc.plan_for_workload(w, ts)
            assert e.value.status == "BC_ERR_NOMEM", str(e.value)
    monkeypatch.delenv("BC_FAULT_INJECT")
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free0 - free1) <= 8 << 20
    # the library still works
    plan = bc.plan_for_workload(w, ts)
    plan.apply(bc.slot_table(ts))
    torch.cuda.synchronize()
    compare(w, [t.cpu().numpy() for t in ts])
