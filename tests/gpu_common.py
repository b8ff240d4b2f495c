"""Shared helpers of the GPU parity tests: run the library and the oracle
on the same seeded inputs and compare element by element."""
import numpy as np

# FP64 per-step tolerance, relative to each field's scale (max |value|)
TOL = 1e-12


def rel_err(a, b, scale=None):
    a, b = np.asarray(a), np.asarray(b)
    s = max(scale if scale is not None else np.max(np.abs(b)), 1e-300)
    return float(np.max(np.abs(a - b)) / s) if a.size else 0.0


def periodic_delta(a, b, L):
    d = a - b
    return (d + 0.5 * L) % L - 0.5 * L


def compare_conserved(gpu, ref, cfg, tol=TOL):
    """Conserved variables and points of the library against the oracle.
    Mass and energy are measured against their own scale; momentum against
    the larger of its own and mass times sound speed: its net value can be
    far below the pressure and advection terms that update it (a shear flow
    with a small transverse seed), whose round-off sets the agreement."""
    a, b = gpu.conserved(), ref.conserved()
    errs = {}
    mscale = float(np.max(np.abs(b["m"])) * np.max(ref.field("cs")))
    for k in ("m", "px", "py", "E"):
        sc = max(float(np.max(np.abs(b[k]))), mscale) if k in ("px", "py") else None
        errs[k] = rel_err(a[k], b[k], sc)
    Lx, Ly = cfg["x1"] - cfg["x0"], cfg["y1"] - cfg["y0"]
    dx = periodic_delta(a["x"], b["x"], Lx) if cfg["boundary"] == 1 else a["x"] - b["x"]
    dy = periodic_delta(a["y"], b["y"], Ly) if cfg["boundary"] == 1 else a["y"] - b["y"]
    errs["x"] = float(np.max(np.abs(dx)) / Lx)
    errs["y"] = float(np.max(np.abs(dy)) / Ly)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (bad, errs)
    return errs


def grad_scale(ref, c):
    """Scale of gradient component c (d/dx, d/dy of rho, vx, vy, p) for the
    parity tolerance.  Eq. 1 sums terms phi_j L_ij / A_i of size |phi| / h,
    so its round-off, and any round-off already in the field values (on a
    moved mesh the densities carry the Section 5 area mismatch, whose
    rounding follows the conditioning of the Voronoi vertices), scales with
    max |phi| / h rather than with the gradient itself; h is the smallest
    cell size sqrt(min A)."""
    import numpy as np
    phi = ref.field(["rho", "vx", "vy", "p"][c // 2])
    h = float(np.sqrt(np.min(ref.field("area"))))
    return max(float(np.max(np.abs(ref.field("grad", c)))), float(np.max(np.abs(phi))) / h)
