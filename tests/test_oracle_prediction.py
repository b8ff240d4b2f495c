"""Pins of the oracle's half-step prediction of the edge states (Section 2.3,
"extrapolated fluxes": the Eq. 2 extrapolation advanced half a step in time
with the primitive Euler equations, in the frame moving with the edge).

What fixes it, independently of the oracle's arithmetic: exact solutions of
the Euler equations that a first-order Taylor step in time reproduces
exactly, or up to a known second-order term.

  A  advected linear density (uniform p and v): rho(x, t) = rho(x - v t);
     the prediction at the moving face point x_f + w_f tau (tau = dt/2) is
     exact.
  B  uniform density and velocity, linear pressure: the fluid accelerates
     uniformly, v(t) = v0 - (b/rho) t, and p(x, t) = p0 + b.(x - v0 t) +
     |b|^2 t^2 / (2 rho); the prediction gets rho and v exactly and p up to
     that t^2 term.
  C  uniform density and pressure, linear velocity v = B0 x (homologous
     flow): B(t) = B0 (I + B0 t)^-1, rho(t) = rho0 / det(I + B0 t),
     p(t) = p0 det(I + B0 t)^-gamma; at the centre of mass the prediction
     differs from this by O(tau^2) in every component, so halving tau
     quarters the error.

Each planted mistake (a dropped term, a wrong sign, a missing gamma, the lab
velocity instead of the velocity relative to the edge, swapped gradient
components) is planted in a copy of the oracle and must fail at least one
of A, B, C.
"""
import numpy as np
import pytest

from planted import build_planted

GAMMA = 5.0 / 3.0


def _pred(O, L):
    return lambda hdt, W, g, off, wf: O.predict(GAMMA, hdt, W, g, off, wf, L=L)


def pin_advected_linear_density(pred):
    """A: exact to round-off for several velocities, face velocities and offsets."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        rho0, p0 = 1.5, 0.8
        a = rng.uniform(-0.4, 0.4, 2)
        v = rng.uniform(-1, 1, 2)
        wf = rng.uniform(-1, 1, 2)
        s = rng.uniform(-0.5, 0.5, 2)        # centre of mass
        off = rng.uniform(-0.05, 0.05, 2)    # face point minus centre of mass
        tau = 0.013
        W = [rho0 + a @ s, v[0], v[1], p0]
        g = [a[0], a[1], 0, 0, 0, 0, 0, 0]
        out = pred(tau, W, g, off, wf)
        xf = s + off + wf * tau
        exact = [rho0 + a @ (xf - v * tau), v[0], v[1], p0]
        if not np.allclose(out, exact, rtol=1e-14, atol=1e-14):
            return False
    return True


def pin_uniform_acceleration(pred):
    """B: rho and v exact, p exact up to the known |b|^2 tau^2 / (2 rho) term."""
    rng = np.random.default_rng(12)
    for _ in range(20):
        rho0, p0 = 1.3, 2.0
        b = rng.uniform(-0.6, 0.6, 2)
        v0 = rng.uniform(-1, 1, 2)
        wf = rng.uniform(-1, 1, 2)
        s = rng.uniform(-0.5, 0.5, 2)
        off = rng.uniform(-0.05, 0.05, 2)
        tau = 0.021
        W = [rho0, v0[0], v0[1], p0 + b @ s]
        g = [0, 0, 0, 0, 0, 0, b[0], b[1]]
        out = pred(tau, W, g, off, wf)
        xf = s + off + wf * tau
        v_t = v0 - b / rho0 * tau
        p_t = p0 + b @ (xf - v0 * tau) + (b @ b) * tau * tau / (2 * rho0)
        exact = [rho0, v_t[0], v_t[1], p_t - (b @ b) * tau * tau / (2 * rho0)]
        if not np.allclose(out, exact, rtol=1e-14, atol=1e-14):
            return False
    return True


def homologous_exact(B0, rho0, p0, x, tau):
    M = np.eye(2) + B0 * tau
    Bt = B0 @ np.linalg.inv(M)
    det = np.linalg.det(M)
    v = Bt @ x
    return np.array([rho0 / det, v[0], v[1], p0 * det ** (-GAMMA)])


def pin_homologous_flow(pred):
    """C: second order in tau against the exact homologous flow (ratio of the
    errors at tau and tau/2 near 4; a first-order mistake gives near 2)."""
    for B0 in (np.array([[0.7, 0.3], [-0.2, 0.4]]), np.array([[-0.5, 0.6], [0.1, -0.3]])):
        rho0, p0 = 1.1, 0.9
        s = np.array([0.3, -0.2])
        wf = np.array([-0.4, 0.25])
        W = [rho0, *(B0 @ s), p0]
        g = [0, 0, B0[0, 0], B0[0, 1], B0[1, 0], B0[1, 1], 0, 0]
        errs = []
        for tau in (0.02, 0.01, 0.005):
            out = pred(tau, W, g, (0.0, 0.0), wf)
            errs.append(np.abs(out - homologous_exact(B0, rho0, p0, s + wf * tau, tau)))
        for c in range(4):
            r1, r2 = errs[0][c] / errs[1][c], errs[1][c] / errs[2][c]
            if not (3.6 < r1 < 4.4 and 3.8 < r2 < 4.2):
                return False
    return True


PINS = (pin_advected_linear_density, pin_uniform_acceleration, pin_homologous_flow)


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_prediction_pins(oracle, pin):
    assert pin(_pred(oracle, None))


def test_homologous_reference_is_an_euler_solution():
    """The closed form used by pin C solves the primitive Euler equations:
    finite differences in time of rho, p and B match -rho tr B, -gamma p tr B
    and -B^2 (no pressure gradient, uniform density)."""
    B0 = np.array([[0.7, 0.3], [-0.2, 0.4]])
    t, h = 0.3, 1e-5
    x = np.array([0.2, 0.1])

    def state(tt):
        M = np.eye(2) + B0 * tt
        return B0 @ np.linalg.inv(M), np.linalg.det(M)

    Bm, dm = state(t - h)
    Bp, dp = state(t + h)
    B, d = state(t)
    dB = (Bp - Bm) / (2 * h)
    np.testing.assert_allclose(dB, -B @ B, rtol=1e-8, atol=1e-9)
    rho = lambda dd: 1.1 / dd
    p = lambda dd: 0.9 * dd ** (-GAMMA)
    np.testing.assert_allclose((rho(dp) - rho(dm)) / (2 * h), -rho(d) * np.trace(B), rtol=1e-8)
    np.testing.assert_allclose((p(dp) - p(dm)) / (2 * h), -GAMMA * p(d) * np.trace(B), rtol=1e-8)
    # the velocity at a fixed point: v_t + (v.grad) v = (B' + B B) x = 0
    np.testing.assert_allclose(dB @ x + B @ (B @ x), 0, atol=1e-9)


# planted mistakes: (name, text in the oracle's predict(), replacement)
MISTAKES = [
    ("drop rho div v", "uy * g[1] + rho * div)", "uy * g[1])"),
    ("drop gamma", "gam * p * div", "p * div"),
    ("sign of grad p / rho", "uy * g[3] + g[6] / rho", "uy * g[3] - g[6] / rho"),
    ("lab velocity, not relative to the edge", "double ux = vx - wf[0], uy = vy - wf[1];",
     "double ux = vx, uy = vy;"),
    ("swapped density gradient components", "ux * g[0] + uy * g[1]", "ux * g[1] + uy * g[0]"),
    ("drop velocity advection", "out[1] -= hdt * (ux * g[2] + uy * g[3] + g[6] / rho);",
     "out[1] -= hdt * (g[6] / rho);"),
    ("drop pressure advection", "out[3] -= hdt * (ux * g[6] + uy * g[7] + gam * p * div);",
     "out[3] -= hdt * (gam * p * div);"),
    ("full step instead of half", "out[0] -= hdt * (", "out[0] -= 2.0 * hdt * ("),
]


@pytest.mark.parametrize("name,old,new", MISTAKES, ids=[m[0] for m in MISTAKES])
def test_planted_mistake_fails_a_pin(oracle, tmp_path, name, old, new):
    L = oracle.load(build_planted(tmp_path, old, new))
    pred = _pred(oracle, L)
    failed = [pin.__name__ for pin in PINS if not pin(pred)]
    assert failed, f"planted mistake '{name}' passes every prediction pin"
