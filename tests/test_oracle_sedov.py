"""The Sedov-Taylor blast in two dimensions (the benchmark's Sedov problem
at 4,096 cells and Courant number 0.03): once the blast wave has swept up
many times the deposited mass, dimensional analysis leaves
R(t) = xi (E t^2 / rho)^(1/4), so every length of the flow grows as t^(1/2)
whatever the similarity constant xi (the constant itself needs the Sedov
energy integral and stays unpinned).  The length measured is the
kinetic-energy-weighted rms radius, which uses every moving cell (the
radius of the few cells compressed past rho = 2 scattered from 0.46 to
0.50 in slope over seeds at this resolution; this one from 0.507 to
0.511).  Also checked: mass and total energy stay constant to round-off
over the whole run (reflective walls).  The scheme has no floor, so the
run must stay clear of the empty blast centre: at 4,096 cells Courant
number 0.05 fails before t = 0.024 on some seeds; 0.03 does not."""
import numpy as np

from paper_1410_3219_gb300 import workloads as W


def kinetic_radius(s, n):
    X, Y, _ = s.points()
    r2 = X[:n] ** 2 + Y[:n] ** 2
    pr, c = s.primitives(), s.conserved()
    ek = c["m"] * (pr["vx"] ** 2 + pr["vy"] ** 2)
    return float(np.sqrt(np.sum(ek * r2) / np.sum(ek)))


def test_blast_grows_as_sqrt_t(oracle):
    n = 4096
    wl = W.sedov(n=n, seed=2)
    wl["cfg"] = dict(wl["cfg"], cfl=0.03)
    s = oracle.Sim(wl)
    c0 = s.conserved()
    R = {}
    # free-running steps (no landing on the sampling times, which would
    # change the run); each radius is taken at the first step past its time
    while s.t < 0.024:
        s.step()
        for t in (0.008, 0.024):
            if t not in R and s.t >= t:
                R[t] = (s.t, kinetic_radius(s, n))
    (ta, ra), (tb, rb) = R[0.008], R[0.024]
    slope = np.log(rb / ra) / np.log(tb / ta)
    assert abs(slope - 0.5) < 0.03, (R, slope)
    c1 = s.conserved()
    for k in ("m", "E"):
        assert abs(np.sum(c1[k]) - np.sum(c0[k])) <= 1e-12 * np.sum(c0[k]), k
