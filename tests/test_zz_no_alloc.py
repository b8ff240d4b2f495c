"""The allocation-free time-step entry point (rich_courant_dt_noalloc).

It exists for callers that cannot allocate GPU memory where they need a time
step: code inside a device memory pool or arena that owns the GPU, and code
where the implicit device synchronisation of an allocation or free is not
allowed.  These tests check, through the C ABI, that two calls in a row
return the same time step as the regular step entry point (rich_step)
computed from the same cell values, within the tolerance of the other parity
tests, for a moving and a static mesh (where the mesh velocity may be NULL);
that it rejects what the other entry points reject; and that a bad cell
shows in the result instead of being skipped.  It lives in a file of its own
that pytest collects last."""
import math

import numpy as np
import pytest

from paper_1410_3219_gb300 import workloads as W
from tests.gpu_common import TOL

pytestmark = pytest.mark.gpu

FIELDS = ("area", "rho", "vx", "vy", "p", "wx", "wy")


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_3219_gb300 import rich
    return rich


@pytest.mark.parametrize("motion", [W.MESH_LAGRANGIAN, W.MESH_EULERIAN])
def test_noalloc_time_step_matches_step_entry_point(motion):
    import torch
    rich = _lib()

    wl = W.sedov(n=20000, seed=12, motion=motion)
    sim = rich.Sim(wl)
    n = sim.n
    stream = torch.cuda.current_stream()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        info = sim.step(1)  # regular entry point: its dt comes from the sweep's own reduction
        fields = {k: torch.tensor(sim.field(k), dtype=torch.float64, device="cuda") for k in FIELDS}
        ptrs = [fields[k].data_ptr() for k in FIELDS]
        if motion == W.MESH_EULERIAN:
            ptrs[5] = ptrs[6] = 0  # a static mesh needs no mesh velocity
        rich.rich_courant_dt_noalloc(wl["cfg"], n, *ptrs, out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        dt = float(out.item())
        assert abs(dt - info["dt_last"]) <= TOL * info["dt_last"], (call, dt, info["dt_last"])
        out.fill_(-1.0)
    sim.close()


def test_noalloc_rejects_bad_sizes_and_configs():
    import torch
    rich = _lib()

    x = torch.ones(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cfg = W.default_cfg()
    ptrs = [x.data_ptr()] * 7
    for bad_n in (0, (1 << 24) + 1):
        with pytest.raises(rich.RichError) as e:
            rich.rich_courant_dt_noalloc(cfg, bad_n, *ptrs, out.data_ptr())
        assert e.value.code == -1
    for bad in (dict(gamma=1.0), dict(cfl=0.0), dict(motion=7)):
        with pytest.raises(rich.RichError) as e:
            rich.rich_courant_dt_noalloc(dict(cfg, **bad), 4, *ptrs, out.data_ptr())
        assert e.value.code == -1
    with pytest.raises(rich.RichError):  # a moving mesh needs wx, wy
        rich.rich_courant_dt_noalloc(cfg, 4, *ptrs[:5], 0, 0, out.data_ptr())


def test_noalloc_bad_cell_gives_nan():
    import torch
    rich = _lib()

    n = 3000
    h = 1.0 / 64
    gamma = 1.4
    area = np.full(n, h * h)
    rho = np.full(n, 1.0)
    p = np.full(n, 1.0)
    v = np.zeros(n)
    cfg = W.default_cfg(gamma=gamma, motion=W.MESH_EULERIAN)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    good = [dev(a) for a in (area, rho, v, v, p)]
    rich.rich_courant_dt_noalloc(cfg, n, *[t.data_ptr() for t in good], 0, 0, out.data_ptr())
    torch.cuda.synchronize()
    expect = cfg["cfl"] * math.sqrt(h * h / math.pi) / math.sqrt(gamma)
    assert abs(float(out.item()) - expect) <= TOL * expect
    p_bad = p.copy()
    p_bad[1234] = -1.0  # negative pressure: NaN sound speed
    bad = [dev(a) for a in (area, rho, v, v, p_bad)]
    rich.rich_courant_dt_noalloc(cfg, n, *[t.data_ptr() for t in bad], 0, 0, out.data_ptr())
    torch.cuda.synchronize()
    assert math.isnan(float(out.item()))
