"""ORACLE (test infrastructure only): ctypes binding of the plain C, FP64,
single-threaded restatement of the paper's scheme in this folder.

Only the tests, the smoke check and the benchmark's CPU baseline load this
module.  It never calls into the CUDA library and the CUDA library never
calls into it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_exact.c", "orc_delaunay.c", "orc_hydro.c"]
LIB = os.path.join(HERE, "liborc.so")

FIELDS = {
    "area": 0, "cx": 1, "cy": 2, "rho": 3, "vx": 4, "vy": 5, "p": 6, "cs": 7,
    "grad": 8, "lgrad": 16, "wx": 24, "wy": 25, "tess": 26, "alpha": 27, "dt": 31,
}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction, no fast-math)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES + ["orc.h"]]
    if not force and os.path.exists(LIB):
        if os.path.getmtime(LIB) >= max(os.path.getmtime(s) for s in srcs):
            return LIB
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", LIB + ".tmp"] + [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


class Config(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("boundary", C.c_int),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("motion", C.c_int), ("chi", C.c_double), ("eta", C.c_double),
                ("theta", C.c_double), ("delta_v", C.c_double), ("delta_p", C.c_double),
                ("limiter", C.c_int), ("scheme", C.c_int)]

    @classmethod
    def from_dict(cls, d):
        c = cls()
        for name, _ in cls._fields_:
            setattr(c, name, d.get(name, 0) if name == "scheme" else d[name])
        return c


_lib = None
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(LIB)
    return _lib


def load(path):
    """ctypes handle of an oracle library built at `path`, with argument
    types set (the tests also load copies built with planted mistakes)."""
    L = C.CDLL(path)
    d = C.c_double
    L.orc_orient.argtypes = [d] * 6
    L.orc_incircle_raw.argtypes = [d] * 8
    L.orc_incircle_sos.argtypes = [d] * 8
    L.orc_delaunay.argtypes = [C.c_int, _D, _D, _I, C.POINTER(_I)]
    L.orc_free.argtypes = [C.c_void_p]
    L.orc_create.argtypes = [C.POINTER(Config), C.c_int, _D, _D, _D, _D, _D, _D, C.POINTER(C.c_void_p)]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_tessellate.argtypes = [C.c_void_p]
    L.orc_sweep.argtypes = [C.c_void_p, d, _D]
    L.orc_step.argtypes = [C.c_void_p, d, _D]
    L.orc_time.argtypes = [C.c_void_p]
    L.orc_time.restype = d
    L.orc_band.argtypes = [C.c_void_p]
    L.orc_band.restype = d
    L.orc_num_points.argtypes = [C.c_void_p]
    L.orc_get_points.argtypes = [C.c_void_p, _D, _D, _I]
    L.orc_ring_total.argtypes = [C.c_void_p]
    L.orc_get_ring.argtypes = [C.c_void_p, _I, _I]
    L.orc_get_conserved.argtypes = [C.c_void_p] + [_D] * 6
    L.orc_get_cells.argtypes = [C.c_void_p, C.c_int, _D]
    L.orc_get_primitives.argtypes = [C.c_void_p] + [_D] * 5
    L.orc_hllc.argtypes = [d, _D, _D, _D]
    L.orc_predict.argtypes = [d, d, _D, _D, d, d, _D, _D]
    L.orc_riemann_exact.argtypes = [d] * 7 + [_D, _D]
    L.orc_riemann_sample.argtypes = [d] * 9 + [d, _D]
    return L


def _dp(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def orient(a, b, c):
    return lib().orc_orient(*a, *b, *c)


def incircle(a, b, c, d, sos=True):
    f = lib().orc_incircle_sos if sos else lib().orc_incircle_raw
    return f(*a, *b, *c, *d)


def delaunay(x, y):
    """Triangles (k, 3) of the tie-broken Delaunay triangulation; ids >= n
    belong to the auxiliary enclosing triangle."""
    x, y = _f64(x), _f64(y)
    nt = C.c_int(0)
    tp = _I()
    rc = lib().orc_delaunay(len(x), _dp(x), _dp(y), C.byref(nt), C.byref(tp))
    if rc != 0:
        raise ValueError(f"oracle delaunay failed ({rc})")
    out = np.ctypeslib.as_array(tp, shape=(nt.value * 3,)).reshape(-1, 3).copy()
    lib().orc_free(tp)
    return out


def hllc(gamma, WL, WR):
    F = np.zeros(4)
    lib().orc_hllc(gamma, _dp(_f64(WL)), _dp(_f64(WR)), _dp(F))
    return F


def predict(gamma, hdt, W, g, off, wf, L=None):
    """Edge state of one side (Section 2.3, extrapolated fluxes): Eq. 2
    extrapolation by `off` from the centre of mass, advanced `hdt` in time
    in the frame moving with `wf`; velocity in the lab frame."""
    out = np.zeros(4)
    (L or lib()).orc_predict(gamma, hdt, _dp(_f64(W)), _dp(_f64(g)), float(off[0]), float(off[1]),
                             _dp(_f64(wf)), _dp(out))
    return out


def riemann_exact(gamma, left, right):
    ps, us = C.c_double(), C.c_double()
    rc = lib().orc_riemann_exact(gamma, *left, *right, C.byref(ps), C.byref(us))
    if rc != 0:
        raise ValueError("vacuum")
    return ps.value, us.value


def riemann_sample(gamma, left, right, ps, us, xi):
    xi = np.atleast_1d(np.asarray(xi, np.float64))
    out = np.zeros((xi.size, 3))
    buf = np.zeros(3)
    for k, v in enumerate(xi):
        lib().orc_riemann_sample(gamma, *left, *right, ps, us, float(v), _dp(buf))
        out[k] = buf
    return out


class OracleError(RuntimeError):
    pass


class Sim:
    """One simulation advanced by the oracle."""

    def __init__(self, wl):
        self.cfg = Config.from_dict(wl["cfg"])
        self.n = len(wl["x"])
        arrs = [_f64(wl[k]) for k in ("x", "y", "rho", "vx", "vy", "p")]
        h = C.c_void_p()
        rc = lib().orc_create(C.byref(self.cfg), self.n, *[_dp(a) for a in arrs], C.byref(h))
        if rc != 0:
            raise OracleError(f"orc_create failed ({rc})")
        self.h = h

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tessellate(self):
        rc = lib().orc_tessellate(self.h)
        if rc != 0:
            raise OracleError(f"orc_tessellate failed ({rc})")

    def sweep(self, t_end=np.inf):
        dt = C.c_double()
        rc = lib().orc_sweep(self.h, t_end, C.byref(dt))
        if rc != 0:
            raise OracleError(f"orc_sweep failed ({rc})")
        return dt.value

    def step(self, t_end=np.inf):
        dt = C.c_double()
        rc = lib().orc_step(self.h, t_end, C.byref(dt))
        if rc != 0:
            raise OracleError(f"orc_step failed ({rc})")
        return dt.value

    @property
    def t(self):
        return lib().orc_time(self.h)

    @property
    def band(self):
        return lib().orc_band(self.h)

    def conserved(self):
        out = [np.zeros(self.n) for _ in range(6)]
        lib().orc_get_conserved(self.h, *[_dp(a) for a in out])
        return dict(zip(("x", "y", "m", "px", "py", "E"), out))

    def field(self, name, comp=0):
        out = np.zeros(self.n)
        rc = lib().orc_get_cells(self.h, FIELDS[name] + comp, _dp(out))
        if rc != 0:
            raise OracleError(f"bad field {name}")
        return out

    def points(self):
        npnt = lib().orc_num_points(self.h)
        X, Y, S = np.zeros(npnt), np.zeros(npnt), np.zeros(npnt, np.int32)
        lib().orc_get_points(self.h, _dp(X), _dp(Y), S.ctypes.data_as(_I))
        return X, Y, S

    def rings(self):
        tot = lib().orc_ring_total(self.h)
        if tot < 0:
            raise OracleError("no current tessellation")
        ptr = np.zeros(self.n + 1, np.int32)
        nb = np.zeros(tot, np.int32)
        lib().orc_get_ring(self.h, ptr.ctypes.data_as(_I), nb.ctypes.data_as(_I))
        return ptr, nb

    def primitives(self):
        """rho, vx, vy, p and area on the current positions (re-tessellates
        if the points moved since the last tessellation)."""
        out = [np.zeros(self.n) for _ in range(5)]
        rc = lib().orc_get_primitives(self.h, *[_dp(a) for a in out])
        if rc != 0:
            raise OracleError(f"orc_get_primitives failed ({rc})")
        return dict(zip(("rho", "vx", "vy", "p", "area"), out))
