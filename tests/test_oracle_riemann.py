"""Oracle pins for the Riemann solvers: HLLC of Section 2.4 (consistency,
upwinding, exact contacts, symmetry, tangential Galilean invariance) and the
exact solver that pins the shock-tube runs (jump conditions, isentropic fans,
tabulated Sod star state)."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def euler_flux(g, W):
    r, u, t, p = W
    E = p / (g - 1) + 0.5 * r * (u * u + t * t)
    return np.array([r * u, r * u * u + p, r * u * t, u * (E + p)])


def test_hllc_consistency(oracle):
    rng = np.random.default_rng(1)
    for _ in range(50):
        W = np.array([rng.uniform(0.1, 3), rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.1, 3)])
        g = rng.choice([1.4, 5 / 3])
        np.testing.assert_allclose(oracle.hllc(g, W, W), euler_flux(g, W), rtol=1e-13, atol=1e-13)


def test_hllc_supersonic_upwind(oracle):
    g = 1.4
    WL = np.array([1.0, 5.0, 0.3, 1.0])   # u - c > 0 on both sides
    WR = np.array([0.5, 4.0, -0.2, 0.7])
    np.testing.assert_array_equal(oracle.hllc(g, WL, WR), euler_flux(g, WL))
    np.testing.assert_array_equal(oracle.hllc(g, WR[[0, 1, 2, 3]] * [1, -1, 1, 1], WL * [1, -1, 1, 1]),
                                  euler_flux(g, WL * [1, -1, 1, 1]))


def test_hllc_resolves_stationary_contact(oracle):
    g = 5 / 3
    WL = np.array([2.0, 0.0, 0.7, 1.5])
    WR = np.array([0.3, 0.0, -0.4, 1.5])
    F = oracle.hllc(g, WL, WR)
    np.testing.assert_allclose(F, [0.0, 1.5, 0.0, 0.0], atol=1e-15)


def test_hllc_mirror_states_have_no_mass_flux(oracle):
    g = 1.4
    for u in (-0.7, 0.0, 0.4, 3.0):
        WL = np.array([1.2, u, 0.3, 0.9])
        WR = np.array([1.2, -u, 0.3, 0.9])
        F = oracle.hllc(g, WL, WR)
        scale = np.max(np.abs(euler_flux(g, WL))) + 1.0
        assert abs(F[0]) < 1e-14 * scale and abs(F[3]) < 1e-14 * scale and abs(F[2]) < 1e-14 * scale


def test_hllc_reflection_symmetry(oracle):
    """Swapping the sides and reversing the normal negates mass and energy
    flux and keeps the normal momentum flux."""
    rng = np.random.default_rng(4)
    flip = np.array([1, -1, 1, 1])
    for _ in range(50):
        WL = np.array([rng.uniform(0.1, 3), rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.1, 3)])
        WR = np.array([rng.uniform(0.1, 3), rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.1, 3)])
        F = oracle.hllc(1.4, WL, WR)
        G = oracle.hllc(1.4, WR * flip, WL * flip)
        np.testing.assert_allclose(G, [-F[0], F[1], -F[2], -F[3]], rtol=1e-12, atol=1e-12)


def test_hllc_tangential_galilean(oracle):
    rng = np.random.default_rng(5)
    for _ in range(50):
        WL = np.array([rng.uniform(0.1, 3), rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.1, 3)])
        WR = np.array([rng.uniform(0.1, 3), rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.1, 3)])
        T = rng.uniform(-3, 3)
        F = oracle.hllc(5 / 3, WL, WR)
        G = oracle.hllc(5 / 3, WL + [0, 0, T, 0], WR + [0, 0, T, 0])
        exp = [F[0], F[1], F[2] + T * F[0], F[3] + T * F[2] + 0.5 * T * T * F[0]]
        np.testing.assert_allclose(G, exp, rtol=1e-12, atol=1e-12)


def _golden_sod():
    d = {}
    with open(os.path.join(GOLDEN, "sod_star_state.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            d[t[0]] = [float(v) for v in t[1:]]
    return d


def test_exact_riemann_sod_star_state(oracle):
    d = _golden_sod()
    ps, us = oracle.riemann_exact(d["gamma"][0], d["left"], d["right"])
    assert abs(ps - d["pstar"][0]) < 5e-6
    assert abs(us - d["ustar"][0]) < 5e-6


PROBLEMS = [
    (1.4, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),        # Sod
    (1.4, (1.0, -2.0, 0.4), (1.0, 2.0, 0.4)),         # two rarefactions
    (1.4, (1.0, 0.0, 1000.0), (1.0, 0.0, 0.01)),      # strong shock
    (5 / 3, (5.99924, 19.5975, 460.894), (5.99242, -6.19633, 46.095)),  # two shocks
    (1.4, (1.0, 0.0, 10.0), (1.0, 0.0, 1.0)),         # paper's 1D shock tube states
]


@pytest.mark.parametrize("g,L,R", PROBLEMS)
def test_exact_riemann_satisfies_jump_and_fan_relations(oracle, g, L, R):
    ps, us = oracle.riemann_exact(g, L, R)
    xi = np.linspace(-30, 30, 60001)
    S = oracle.riemann_sample(g, L, R, ps, us, xi)
    rho, u, p = S[:, 0], S[:, 1], S[:, 2]
    # pressure and velocity continuous at the contact (xi = u*)
    k = np.searchsorted(xi, us)
    assert abs(p[k - 1] - p[k + 1]) < 1e-9 * max(ps, 1) and abs(u[k - 1] - u[k + 1]) < 1e-9 * max(abs(us), 1)
    # locate jumps: a shock is a jump in every variable with compression
    jumps = np.where(np.abs(np.diff(rho)) > 1e-6 * rho.max())[0]
    nshock = 0
    for j in jumps:
        a, b = j, j + 1
        r1, u1, p1 = rho[a], u[a], p[a]
        r2, u2, p2 = rho[b], u[b], p[b]
        # a shock jumps by O(1) in both density and pressure between two samples;
        # a contact keeps the pressure, fan samples change by O(sample spacing)
        if abs(p2 - p1) < 1e-2 * max(p1, p2) or abs(r2 - r1) < 1e-2 * max(r1, r2):
            continue
        # Rankine-Hugoniot: shock speed from mass, then momentum and energy balance
        Ssh = (r2 * u2 - r1 * u1) / (r2 - r1)
        mom = (r2 * u2 * (u2 - Ssh) + p2) - (r1 * u1 * (u1 - Ssh) + p1)
        E1 = p1 / (g - 1) + 0.5 * r1 * u1 * u1
        E2 = p2 / (g - 1) + 0.5 * r2 * u2 * u2
        en = ((E2 + p2) * u2 - E2 * Ssh) - ((E1 + p1) * u1 - E1 * Ssh)
        scale = max(p1, p2, r1 * u1 * u1, r2 * u2 * u2)
        assert abs(mom) < 1e-9 * scale
        assert abs(en) < 1e-9 * scale * (abs(u1) + abs(u2) + abs(Ssh) + 1)
        assert abs(Ssh - 0.5 * (xi[a] + xi[b])) < 2 * (xi[1] - xi[0])
        nshock += 1
    assert nshock == (ps > L[2]) + (ps > R[2])
    # inside rarefaction fans: isentropic, Riemann invariant constant, xi = u -/+ c
    c = np.sqrt(g * p / rho)
    ent = p / rho ** g
    for side, (r0, u0, p0) in (("L", L), ("R", R)):
        c0 = np.sqrt(g * p0 / r0)
        if side == "L" and ps < p0:
            fan = (xi > u0 - c0 + 1e-3) & (xi < us - np.sqrt(g * ps / (r0 * (ps / p0) ** (1 / g))) - 1e-3)
            if fan.any():
                np.testing.assert_allclose(ent[fan], p0 / r0 ** g, rtol=1e-11)
                np.testing.assert_allclose(u[fan] + 2 * c[fan] / (g - 1), u0 + 2 * c0 / (g - 1), rtol=1e-11, atol=1e-11)
                np.testing.assert_allclose(u[fan] - c[fan], xi[fan], atol=1e-10)
        if side == "R" and ps < p0:
            fan = (xi < u0 + c0 - 1e-3) & (xi > us + np.sqrt(g * ps / (r0 * (ps / p0) ** (1 / g))) + 1e-3)
            if fan.any():
                np.testing.assert_allclose(ent[fan], p0 / r0 ** g, rtol=1e-11)
                np.testing.assert_allclose(u[fan] - 2 * c[fan] / (g - 1), u0 - 2 * c0 / (g - 1), rtol=1e-11, atol=1e-11)
                np.testing.assert_allclose(u[fan] + c[fan], xi[fan], atol=1e-10)
