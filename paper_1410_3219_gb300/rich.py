"""Thin ctypes binding of librich.so (include/rich.h).

The functions carry the names of the C entry points and only marshal
arguments; every step of the sweep runs in the library's CUDA kernels.  The
library is loaded on first use; if it is missing, or the machine has no CUDA
device, the calls raise instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librich.so")

RICH_OK = 0
RICH_EINVAL, RICH_EDUPLICATE, RICH_ETESS, RICH_ETOOFEW = -1, -2, -3, -4
RICH_ENEGATIVE, RICH_ENAN, RICH_ENOMEM, RICH_ECUDA, RICH_ENODEV, RICH_ESTATE = -5, -6, -7, -8, -9, -10
ERRORS = {-1: "EINVAL", -2: "EDUPLICATE", -3: "ETESS", -4: "ETOOFEW", -5: "ENEGATIVE", -6: "ENAN",
          -7: "ENOMEM", -8: "ECUDA", -9: "ENODEV", -10: "ESTATE"}

FIELDS = {"area": 0, "cx": 1, "cy": 2, "rho": 3, "vx": 4, "vy": 5, "p": 6, "cs": 7, "grad": 8,
          "lgrad": 16, "wx": 24, "wy": 25, "tess": 26, "alpha": 27, "dt": 31}

# names of every entry point declared in include/rich.h
EXPORTS = ["rich_default_config", "rich_init_mesh", "rich_step", "rich_get_state", "rich_get_conserved",
           "rich_destroy", "rich_strerror", "rich_last_error", "rich_set_stream", "rich_tessellate",
           "rich_sweep", "rich_sync", "rich_get_field", "rich_num_cells", "rich_delaunay_host",
           "rich_rings_host", "rich_set_profiling", "rich_kernel_times", "rich_kernel_name",
           "rich_courant_dt_noalloc", "rich_set_diagnostics", "rich_batch_create", "rich_batch_add",
           "rich_batch_step", "rich_batch_query", "rich_batch_get_conserved", "rich_batch_remove",
           "rich_batch_set_diagnostics", "rich_batch_cells", "rich_batch_destroy", "rich_batch_set_launch",
           "rich_batch_launch_info", "rich_server_create", "rich_server_submit", "rich_server_tick",
           "rich_server_query", "rich_server_fetch", "rich_server_batch", "rich_server_destroy",
           "rich_init_conserved", "rich_get_order", "rich_time", "rich_mesh_update_check",
           "rich_probe_pipe_peaks", "rich_batch_inject_barrier_timeout", "rich_server_start",
           "rich_server_stats", "rich_edge_list_check", "rich_tess_phases"]

REQ_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed"}

SIM_STATES = {0: "pending", 1: "running", 2: "done", 3: "failed"}


class RichError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class rich_config(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("boundary", C.c_int32),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("motion", C.c_int32), ("chi", C.c_double), ("eta", C.c_double),
                ("theta", C.c_double), ("delta_v", C.c_double), ("delta_p", C.c_double),
                ("limiter", C.c_int32), ("scheme", C.c_int32), ("precision", C.c_int32)]

    @classmethod
    def from_dict(cls, d):
        c = cls()
        _lib().rich_default_config(C.byref(c))
        for name, _ in cls._fields_:
            if name in d:
                setattr(c, name, d[name])
        return c


class rich_step_info(C.Structure):
    _fields_ = [("steps_done", C.c_int64), ("t", C.c_double), ("dt_last", C.c_double),
                ("sweep_ms", C.c_double), ("tess_ms", C.c_double), ("copy_ms", C.c_double),
                ("n_ghost", C.c_int64), ("n_tri", C.c_int64), ("n_edges", C.c_int64), ("n_slots", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_D = C.POINTER(C.c_double)
_handle = None


def _lib():
    global _handle
    if _handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P, I64, I32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        L.rich_default_config.argtypes = [C.POINTER(rich_config)]
        L.rich_default_config.restype = None
        L.rich_init_mesh.argtypes = [C.POINTER(rich_config), I64] + [_D] * 6 + [C.POINTER(P)]
        L.rich_step.argtypes = [P, I32, d, C.POINTER(rich_step_info)]
        L.rich_get_state.argtypes = [P, I64] + [_D] * 7
        L.rich_get_conserved.argtypes = [P, I64] + [_D] * 6
        L.rich_destroy.argtypes = [P]
        L.rich_destroy.restype = None
        L.rich_strerror.argtypes = [C.c_int]
        L.rich_strerror.restype = C.c_char_p
        L.rich_last_error.argtypes = []
        L.rich_last_error.restype = C.c_char_p
        L.rich_set_stream.argtypes = [P, P]
        L.rich_tessellate.argtypes = [P, C.POINTER(rich_step_info)]
        L.rich_sweep.argtypes = [P, d]
        L.rich_sync.argtypes = [P, C.POINTER(rich_step_info)]
        L.rich_get_field.argtypes = [P, I32, I64, _D]
        L.rich_num_cells.argtypes = [P]
        L.rich_num_cells.restype = I64
        L.rich_delaunay_host.argtypes = [I64, _D, _D, I64, C.POINTER(C.c_int32), C.POINTER(I64)]
        L.rich_mesh_update_check.argtypes = [C.POINTER(rich_config), I64, I32, _D, _D, I32, C.POINTER(C.c_int32),
                                             C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)]
        L.rich_rings_host.argtypes = [C.POINTER(rich_config), I64, _D, _D, I64, C.POINTER(I64), _D, _D,
                                      C.POINTER(I64), C.POINTER(I64)]
        L.rich_set_profiling.argtypes = [P, I32]
        L.rich_set_diagnostics.argtypes = [P, I32]
        L.rich_batch_create.argtypes = [I32, I64, I32, C.POINTER(P)]
        L.rich_batch_add.argtypes = [P, C.POINTER(rich_config), I64] + [_D] * 6 + [d, I64, C.POINTER(I32)]
        L.rich_batch_step.argtypes = [P, C.POINTER(rich_step_info)]
        L.rich_batch_query.argtypes = [P, I32, C.POINTER(I32), C.POINTER(I32), _D, C.POINTER(I64), _D]
        L.rich_batch_get_conserved.argtypes = [P, I32, I64] + [_D] * 6
        L.rich_batch_remove.argtypes = [P, I32]
        L.rich_batch_set_diagnostics.argtypes = [P, I32]
        L.rich_batch_cells.argtypes = [P]
        L.rich_batch_cells.restype = I64
        L.rich_batch_destroy.argtypes = [P]
        L.rich_batch_destroy.restype = None
        L.rich_batch_set_launch.argtypes = [P, I32, I32]
        L.rich_batch_launch_info.argtypes = [P] + [C.POINTER(I32)] * 5 + [C.POINTER(I64)]
        L.rich_server_create.argtypes = [I32, I64, I32, C.POINTER(P)]
        L.rich_server_submit.argtypes = [P, C.POINTER(rich_config), I64] + [_D] * 6 + [d, I64, C.POINTER(I64)]
        L.rich_server_tick.argtypes = [P, C.POINTER(rich_step_info)] + [C.POINTER(I32)] * 3
        L.rich_server_query.argtypes = [P, I64, C.POINTER(I32), C.POINTER(I32), C.POINTER(I64), _D, _D]
        L.rich_server_fetch.argtypes = [P, I64, I64] + [_D] * 6
        L.rich_server_batch.argtypes = [P]
        L.rich_server_batch.restype = P
        L.rich_server_destroy.argtypes = [P]
        L.rich_server_destroy.restype = None
        L.rich_kernel_times.argtypes = [P, I32, _D, C.POINTER(I32)]
        L.rich_kernel_name.argtypes = [I32]
        L.rich_kernel_name.restype = C.c_char_p
        L.rich_courant_dt_noalloc.argtypes = [C.POINTER(rich_config), I64] + [P] * 8 + [P]
        L.rich_init_conserved.argtypes = [C.POINTER(rich_config), I64] + [_D] * 6 + [d, C.POINTER(I64),
                                                                                     C.POINTER(P)]
        L.rich_get_order.argtypes = [P, I64, C.POINTER(I64)]
        L.rich_time.argtypes = [P]
        L.rich_time.restype = d
        L.rich_probe_pipe_peaks.argtypes = [_D, _D]
        L.rich_batch_inject_barrier_timeout.argtypes = [P, I32, C.POINTER(I64)]
        L.rich_server_start.argtypes = [P, I32, I64, I64]
        L.rich_tess_phases.argtypes = [P, _D]
        L.rich_edge_list_check.argtypes = [C.POINTER(rich_config), I64, _D, _D, C.POINTER(I64), C.POINTER(I64)]
        L.rich_server_stats.argtypes = [P, C.POINTER(I64)] + [_D] * 4
        _handle = L
    return _handle


def lib():
    return _lib()


def _check(rc):
    if rc != RICH_OK:
        raise RichError(rc, _lib().rich_last_error().decode())
    return rc


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.shape != (n,):
        raise ValueError("bad array shape")
    return a


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


# ---- the C entry points -----------------------------------------------------

def rich_init_mesh(cfg, x, y, rho, vx, vy, p):
    c = cfg if isinstance(cfg, rich_config) else rich_config.from_dict(cfg)
    n = len(x)
    arrs = [_f64(a, n) for a in (x, y, rho, vx, vy, p)]
    h = C.c_void_p()
    _check(_lib().rich_init_mesh(C.byref(c), n, *[_p(a) for a in arrs], C.byref(h)))
    return h


def rich_init_conserved(cfg, x, y, m, px, py, E, t=0.0, order=None):
    c = cfg if isinstance(cfg, rich_config) else rich_config.from_dict(cfg)
    n = len(x)
    arrs = [_f64(a, n) for a in (x, y, m, px, py, E)]
    o = None
    if order is not None:
        o = np.ascontiguousarray(order, dtype=np.int64)
        if o.shape != (n,):
            raise ValueError("order must have one entry per point")
    h = C.c_void_p()
    _check(_lib().rich_init_conserved(C.byref(c), n, *[_p(a) for a in arrs], float(t),
                                      o.ctypes.data_as(C.POINTER(C.c_int64)) if o is not None else None,
                                      C.byref(h)))
    return h


def rich_get_order(h, n):
    o = np.empty(n, np.int64)
    _check(_lib().rich_get_order(h, n, o.ctypes.data_as(C.POINTER(C.c_int64))))
    return o


def rich_time(h):
    return _lib().rich_time(h)


def rich_step(h, max_steps=1, t_end=float("inf")):
    info = rich_step_info()
    _check(_lib().rich_step(h, max_steps, t_end, C.byref(info)))
    return info.as_dict()


def rich_get_state(h, n):
    out = [np.zeros(n) for _ in range(7)]
    _check(_lib().rich_get_state(h, n, *[_p(a) for a in out]))
    return dict(zip(("x", "y", "rho", "vx", "vy", "p", "area"), out))


def rich_get_conserved(h, n):
    out = [np.zeros(n) for _ in range(6)]
    _check(_lib().rich_get_conserved(h, n, *[_p(a) for a in out]))
    return dict(zip(("x", "y", "m", "px", "py", "E"), out))


def rich_destroy(h):
    _lib().rich_destroy(h)


def rich_set_stream(h, stream_ptr):
    _check(_lib().rich_set_stream(h, C.c_void_p(stream_ptr)))


def rich_tessellate(h):
    info = rich_step_info()
    _check(_lib().rich_tessellate(h, C.byref(info)))
    return info.as_dict()


def rich_sweep(h, t_end=float("inf")):
    _check(_lib().rich_sweep(h, t_end))


def rich_sync(h):
    info = rich_step_info()
    _check(_lib().rich_sync(h, C.byref(info)))
    return info.as_dict()


def rich_get_field(h, n, name, comp=0):
    out = np.zeros(n)
    _check(_lib().rich_get_field(h, FIELDS[name] + comp, n, _p(out)))
    return out


def rich_set_diagnostics(h, on=True):
    _check(_lib().rich_set_diagnostics(h, 1 if on else 0))


def rich_set_profiling(h, on=True):
    _check(_lib().rich_set_profiling(h, 1 if on else 0))


def rich_kernel_times(h):
    ms = np.zeros(16)
    cnt = C.c_int32()
    _check(_lib().rich_kernel_times(h, 16, _p(ms), C.byref(cnt)))
    return {rich_kernel_name(k): float(ms[k]) for k in range(cnt.value)}


def rich_kernel_name(k):
    return _lib().rich_kernel_name(k).decode()


def rich_courant_dt_noalloc(cfg, n, area, rho, vx, vy, p, wx, wy, dt_out, stream=0):
    """Device pointers (ints) in, device pointer out; see include/rich.h."""
    c = cfg if isinstance(cfg, rich_config) else rich_config.from_dict(cfg)
    ptrs = [C.c_void_p(v) if v else None for v in (area, rho, vx, vy, p, wx, wy, dt_out)]
    _check(_lib().rich_courant_dt_noalloc(C.byref(c), n, *ptrs, C.c_void_p(stream)))


def rich_probe_pipe_peaks():
    """Measured FP64 and FP32 FMA-chain peaks of the current device (TFLOP/s)."""
    a, b = C.c_double(), C.c_double()
    _check(_lib().rich_probe_pipe_peaks(C.byref(a), C.byref(b)))
    return a.value, b.value


def rich_tess_phases(h):
    """Wall time (ms) of the phases of the last host tessellation: ghosts and
    grid, tiles, assembly, edges and order."""
    ms = np.zeros(4)
    _check(_lib().rich_tess_phases(h, _p(ms)))
    return dict(zip(("ghosts_grid", "tiles", "assembly", "edges_order"), ms.tolist()))


def rich_edge_list_check(cfg, x, y):
    """(edges, mismatched entries) of the device edge-list builder against
    the host's on the same rings."""
    c = cfg if isinstance(cfg, rich_config) else rich_config.from_dict(cfg)
    x, y = _f64(x), _f64(y)
    e, m = C.c_int64(), C.c_int64()
    _check(_lib().rich_edge_list_check(C.byref(c), len(x), _p(x), _p(y), C.byref(e), C.byref(m)))
    return e.value, m.value


def rich_delaunay_host(x, y):
    x, y = _f64(x), _f64(y)
    n = len(x)
    cap = 2 * n + 16
    tris = np.zeros(3 * cap, np.int32)
    nt = C.c_int64()
    _check(_lib().rich_delaunay_host(n, _p(x), _p(y), cap, tris.ctypes.data_as(C.POINTER(C.c_int32)),
                                     C.byref(nt)))
    return tris[:3 * nt.value].reshape(-1, 3)


def rich_rings_host(cfg, x, y):
    c = cfg if isinstance(cfg, rich_config) else rich_config.from_dict(cfg)
    x, y = _f64(x), _f64(y)
    n = len(x)
    ptr = np.zeros(n + 1, np.int64)
    ns = C.c_int64()
    cap = 12 * n + 64
    nbx, nby, src = np.zeros(cap), np.zeros(cap), np.zeros(cap, np.int64)
    I64P = C.POINTER(C.c_int64)
    _check(_lib().rich_rings_host(C.byref(c), n, _p(x), _p(y), cap, ptr.ctypes.data_as(I64P), _p(nbx), _p(nby),
                                  src.ctypes.data_as(I64P), C.byref(ns)))
    k = ns.value
    return ptr, nbx[:k], nby[:k], src[:k]


def rich_mesh_update_check(cfg, xs, ys, threads=4):
    """Host meshes of successive point sets (rows of the 2D arrays xs, ys)
    built with one reused workspace and afresh: (steps whose sweep inputs
    differ, tiles updated in place, tiles rebuilt, vertices taken out and
    re-inserted by the updates)."""
    c = cfg if isinstance(cfg, rich_config) else rich_config.from_dict(cfg)
    xs, ys = np.atleast_2d(xs), np.atleast_2d(ys)
    steps, n = xs.shape
    xs, ys = _f64(xs.ravel()), _f64(ys.ravel())
    mis, up, re, ri = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int64()
    _check(_lib().rich_mesh_update_check(C.byref(c), n, steps, _p(xs), _p(ys), threads, C.byref(mis), C.byref(up),
                                         C.byref(re), C.byref(ri)))
    return mis.value, up.value, re.value, ri.value



def rich_batch_create(precision=0, max_cells=1 << 24, host_threads=0):
    h = C.c_void_p()
    _check(_lib().rich_batch_create(precision, max_cells, host_threads, C.byref(h)))
    return h


def rich_batch_add(b, cfg, x, y, rho, vx, vy, p, t_end=float("inf"), max_steps=1 << 62):
    c = cfg if isinstance(cfg, rich_config) else rich_config.from_dict(cfg)
    n = len(x)
    arrs = [_f64(a, n) for a in (x, y, rho, vx, vy, p)]
    sid = C.c_int32()
    _check(_lib().rich_batch_add(b, C.byref(c), n, *[_p(a) for a in arrs], t_end, max_steps, C.byref(sid)))
    return sid.value


def rich_batch_step(b):
    info = rich_step_info()
    _check(_lib().rich_batch_step(b, C.byref(info)))
    return info.as_dict()


def rich_batch_query(b, sid):
    st, err, t, steps, lat = C.c_int32(), C.c_int32(), C.c_double(), C.c_int64(), C.c_double()
    _check(_lib().rich_batch_query(b, sid, C.byref(st), C.byref(err), C.byref(t), C.byref(steps), C.byref(lat)))
    return {"state": SIM_STATES.get(st.value, st.value), "error": err.value, "t": t.value, "steps": steps.value,
            "latency_ms": lat.value}


def rich_batch_get_conserved(b, sid, n):
    out = [np.zeros(n) for _ in range(6)]
    _check(_lib().rich_batch_get_conserved(b, sid, n, *[_p(a) for a in out]))
    return dict(zip(("x", "y", "m", "px", "py", "E"), out))


def rich_batch_remove(b, sid):
    _check(_lib().rich_batch_remove(b, sid))


def rich_batch_set_diagnostics(b, on=True):
    _check(_lib().rich_batch_set_diagnostics(b, 1 if on else 0))


def rich_batch_cells(b):
    return _lib().rich_batch_cells(b)


def rich_batch_set_launch(b, mode=0, block=256):
    _check(_lib().rich_batch_set_launch(b, mode, block))


def rich_batch_launch_info(b):
    v = [C.c_int32() for _ in range(5)]
    cnt = (C.c_int64 * 4)()
    _check(_lib().rich_batch_launch_info(b, *[C.byref(x) for x in v], cnt))
    return {"persistent": v[0].value, "block": v[1].value, "grid": v[2].value, "tuned": v[3].value,
            "graph": v[4].value, "staged_steps": cnt[0], "persistent_steps": cnt[1], "graph_replays": cnt[2],
            "graph_recordings": cnt[3]}


def rich_batch_destroy(b):
    _lib().rich_batch_destroy(b)


class Batch:
    """Many independent simulations stepped together (device-resident)."""

    def __init__(self, precision=0, max_cells=1 << 24, host_threads=0):
        self.h = rich_batch_create(precision, max_cells, host_threads)
        self.sizes = {}

    def add(self, wl, t_end=float("inf"), max_steps=1 << 62):
        sid = rich_batch_add(self.h, wl["cfg"], wl["x"], wl["y"], wl["rho"], wl["vx"], wl["vy"], wl["p"],
                             t_end, max_steps)
        self.sizes[sid] = len(wl["x"])
        return sid

    def step(self):
        return rich_batch_step(self.h)

    def query(self, sid):
        return rich_batch_query(self.h, sid)

    def conserved(self, sid):
        return rich_batch_get_conserved(self.h, sid, self.sizes[sid])

    def remove(self, sid):
        rich_batch_remove(self.h, sid)

    def set_launch(self, mode=0, block=256):
        rich_batch_set_launch(self.h, mode, block)

    def launch_info(self):
        return rich_batch_launch_info(self.h)

    def inject_barrier_timeout(self, spin_limit=0):
        """Arm (spin_limit > 0) a barrier timeout in the next persistent
        sweep; returns the number of timed-out persistent sweeps so far."""
        seen = C.c_int64()
        _check(_lib().rich_batch_inject_barrier_timeout(self.h, spin_limit, C.byref(seen)))
        return seen.value

    def close(self):
        if self.h:
            rich_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (native scheduler in librich.so)."""

    def __init__(self, precision=0, max_cells=1 << 24, host_threads=0):
        h = C.c_void_p()
        _check(_lib().rich_server_create(precision, max_cells, host_threads, C.byref(h)))
        self.h = h
        self.sizes = {}

    def submit(self, wl, t_end=float("inf"), max_steps=1 << 62):
        c = rich_config.from_dict(wl["cfg"])
        n = len(wl["x"])
        arrs = [_f64(wl[k], n) for k in ("x", "y", "rho", "vx", "vy", "p")]
        rid = C.c_int64()
        _check(_lib().rich_server_submit(self.h, C.byref(c), n, *[_p(a) for a in arrs], t_end, max_steps,
                                         C.byref(rid)))
        self.sizes[rid.value] = n
        return rid.value

    def tick(self):
        info = rich_step_info()
        a, r, q = C.c_int32(), C.c_int32(), C.c_int32()
        _check(_lib().rich_server_tick(self.h, C.byref(info), C.byref(a), C.byref(r), C.byref(q)))
        out = info.as_dict()
        out.update(admitted=a.value, running=r.value, queued=q.value)
        return out

    def query(self, rid):
        st, err, steps, qm, lm = C.c_int32(), C.c_int32(), C.c_int64(), C.c_double(), C.c_double()
        _check(_lib().rich_server_query(self.h, rid, C.byref(st), C.byref(err), C.byref(steps), C.byref(qm),
                                        C.byref(lm)))
        return {"state": REQ_STATES.get(st.value, st.value), "error": err.value, "steps": steps.value,
                "queue_ms": qm.value, "latency_ms": lm.value}

    def fetch(self, rid):
        n = self.sizes.pop(rid)
        out = [np.zeros(n) for _ in range(6)]
        _check(_lib().rich_server_fetch(self.h, rid, n, *[_p(a) for a in out]))
        return dict(zip(("x", "y", "m", "px", "py", "E"), out))

    def launch_info(self):
        return rich_batch_launch_info(_lib().rich_server_batch(self.h))

    def start(self, lanes=2, split_cells=65536, top_lane_cells=0):
        """Asynchronous mode: lane threads step the requests (see rich.h)."""
        _check(_lib().rich_server_start(self.h, lanes, split_cells, top_lane_cells))

    def stats(self):
        st = C.c_int64()
        v = [C.c_double() for _ in range(4)]
        _check(_lib().rich_server_stats(self.h, C.byref(st), *[C.byref(x) for x in v]))
        return {"steps": st.value, "sweep_ms": v[0].value, "tess_ms": v[1].value, "other_ms": v[2].value,
                "wall_ms": v[3].value}

    def close(self):
        if self.h:
            _lib().rich_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- convenience wrapper ------------------------------------------------------

class Sim:
    """One simulation owned by the library (device-resident state)."""

    def __init__(self, wl):
        self.n = len(wl["x"])
        self.h = rich_init_mesh(wl["cfg"], wl["x"], wl["y"], wl["rho"], wl["vx"], wl["vy"], wl["p"])

    def close(self):
        if self.h:
            rich_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, max_steps=1, t_end=float("inf")):
        return rich_step(self.h, max_steps, t_end)

    def tessellate(self):
        return rich_tessellate(self.h)

    def sweep(self, t_end=float("inf")):
        rich_sweep(self.h, t_end)

    def sync(self):
        return rich_sync(self.h)

    def set_stream(self, ptr):
        rich_set_stream(self.h, ptr)

    def state(self):
        return rich_get_state(self.h, self.n)

    def conserved(self):
        return rich_get_conserved(self.h, self.n)

    def checkpoint(self):
        """Everything a bit-identical restart needs (take it between steps)."""
        c = rich_get_conserved(self.h, self.n)
        c["t"] = rich_time(self.h)
        c["order"] = rich_get_order(self.h, self.n)
        return c

    @classmethod
    def restart(cls, cfg, ck):
        """A simulation continuing from checkpoint() output."""
        self = cls.__new__(cls)
        self.n = len(ck["x"])
        self.h = rich_init_conserved(cfg, ck["x"], ck["y"], ck["m"], ck["px"], ck["py"], ck["E"], ck["t"],
                                     ck.get("order"))
        return self

    def field(self, name, comp=0):
        return rich_get_field(self.h, self.n, name, comp)
