"""Checkpoint and restart through the C ABI (rich_get_conserved + rich_time
+ rich_get_order, then rich_init_conserved): a simulation restarted from a
checkpoint taken between steps repeats the uninterrupted run bit for bit,
in both precisions and both time advancements; without the cell order the
restart is valid but renumbers the cells, so it agrees to round-off only.
The paper has no checkpoint facility; this is the framework's own."""
import numpy as np
import pytest

from paper_1410_3219_gb300 import workloads as W
from tests.gpu_common import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_3219_gb300 import rich
    return rich


def variant(make, precision=W.FP64, scheme=W.SCHEME_EXTRAPOLATED):
    wl = make()
    wl["cfg"]["precision"] = precision
    wl["cfg"]["scheme"] = scheme
    return wl


CASES = {
    "sedov_fp64": lambda: variant(lambda: W.sedov(n=4096)),
    "kh_split": lambda: variant(lambda: W.kelvin_helmholtz(n_side=48, amp=0.1), precision=W.FP32_SPLIT),
    "gresho_time_centred": lambda: variant(lambda: W.gresho(n_side=32), scheme=W.SCHEME_TIME_CENTRED),
    "mixed_walls_split_time_centred": lambda: variant(lambda: W.random_mixed(n=1500, seed=8),
                                                      precision=W.FP32_SPLIT, scheme=W.SCHEME_TIME_CENTRED),
}


@pytest.mark.parametrize("name", list(CASES))
def test_restart_is_bit_identical(R, name):
    wl = CASES[name]()
    a = R.Sim(wl)
    a.step(5)
    ck = a.checkpoint()
    ia = a.step(5)
    b = R.Sim.restart(wl["cfg"], ck)
    ib = b.step(5)
    assert ia["steps_done"] == ib["steps_done"] == 5
    assert ia["t"] == ib["t"]
    ca, cb = a.conserved(), b.conserved()
    for k in ("x", "y", "m", "px", "py", "E"):
        assert np.array_equal(ca[k], cb[k]), k
    a.close()
    b.close()


def test_restart_without_order_agrees_to_round_off(R):
    wl = CASES["sedov_fp64"]()
    a = R.Sim(wl)
    a.step(3)
    ck = a.checkpoint()
    ck.pop("order")
    a.step(3)
    b = R.Sim.restart(wl["cfg"], ck)
    b.step(3)
    ca, cb = a.conserved(), b.conserved()
    for k in ("m", "px", "py", "E"):
        assert rel_err(cb[k], ca[k]) <= 1e-12, k
    a.close()
    b.close()


def test_restart_rejects_bad_input(R):
    wl = W.sod(n_side=16)
    a = R.Sim(wl)
    ck = a.checkpoint()
    bad = dict(ck, order=np.zeros(len(ck["x"]), np.int64))
    with pytest.raises(R.RichError):
        R.Sim.restart(wl["cfg"], bad)
    neg = dict(ck, m=-ck["m"])
    with pytest.raises(R.RichError):
        R.Sim.restart(wl["cfg"], neg)
    a.close()
