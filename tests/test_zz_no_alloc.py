"""The allocation-free time-step entry point (rich_courant_dt_noalloc).

It exists for callers that cannot allocate GPU memory where they need a time
step (inside a device memory pool or arena, where an allocation's implicit
synchronisation is not allowed, or in launch sequences recorded for replay).
This test checks, through the C ABI, that two calls in a row return the same
time step as the regular step entry point (rich_step) computed from the same
cell values, within the tolerance of the other parity tests.  It lives in a
file of its own that pytest collects last."""
import numpy as np
import pytest

from paper_1410_3219_gb300 import workloads as W
from tests.gpu_common import TOL

pytestmark = pytest.mark.gpu


def test_noalloc_time_step_matches_step_entry_point():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_3219_gb300 import rich

    wl = W.sedov(n=20000, seed=12)
    sim = rich.Sim(wl)
    n = sim.n
    stream = torch.cuda.current_stream()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        info = sim.step(1)  # regular entry point: its dt comes from the sweep's own reduction
        fields = {k: torch.tensor(sim.field(k), dtype=torch.float64, device="cuda")
                  for k in ("area", "rho", "vx", "vy", "p", "wx", "wy")}
        rich.rich_courant_dt_noalloc(wl["cfg"], n, *[fields[k].data_ptr() for k in
                                                     ("area", "rho", "vx", "vy", "p", "wx", "wy")],
                                     out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        dt = float(out.item())
        assert abs(dt - info["dt_last"]) <= TOL * info["dt_last"], (call, dt, info["dt_last"])
        out.fill_(-1.0)
    sim.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_3219_gb300 import rich

    x = torch.ones(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cfg = W.default_cfg()
    ptrs = [x.data_ptr()] * 7
    for bad_n in (0, (1 << 24) + 1):
        with pytest.raises(rich.RichError) as e:
            rich.rich_courant_dt_noalloc(cfg, bad_n, *ptrs, out.data_ptr())
        assert e.value.code == -1
