"""FP64 CPU oracle for the shallow-water finite-volume step.

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, obviously-correct
statement of the method in Sections 2-3 of Delmas & Soulaimani (Eq 1-37):
HLLC fluxes with the adaptive h* estimate, hydrostatic reconstruction of the
bed source, semi-implicit Manning friction, explicit Euler with the CFL
condition on the inscribed radius.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA library under ``paper_2010_14416_gb300/``.

The C source is ``swe_oracle.c`` (compiled on first use with gcc, FMA
contraction off, OpenMP over cells).  This module is argument marshalling.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swe_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC_WALL, BC_INFLOW, BC_TRANSMISSIVE, BC_STAGE = 0, 1, 2, 3
G_DEFAULT = 9.81
H_DRY_DEFAULT = 1e-6


def build(force: bool = False) -> str:
    """Compiles the oracle's C source into a shared library (in-tree)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_LIB_PATH)
        dp, ip, lp = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
        vp = C.c_void_p
        lib.orc_mesh_new.restype = vp
        lib.orc_mesh_new.argtypes = [dp, C.c_int64, ip, C.c_int64, dp, dp, C.c_double,
                                     C.c_double, C.POINTER(C.c_int)]
        lib.orc_mesh_free.argtypes = [vp]
        lib.orc_mesh_set_bc.restype = C.c_int
        lib.orc_mesh_set_bc.argtypes = [vp, ip, C.c_int64, C.c_int, C.c_double]
        lib.orc_mesh_geometry.argtypes = [vp, dp, dp, lp, dp, dp, dp]
        lib.orc_mesh_set_fields.argtypes = [vp, dp, dp]
        lib.orc_boundary_discharge.restype = C.c_int
        lib.orc_boundary_discharge.argtypes = [vp, dp, dp, dp, dp]
        lib.orc_mesh_groups.restype = C.c_int
        lib.orc_mesh_groups.argtypes = [vp, C.POINTER(C.c_int), dp, dp]
        lib.orc_hstar.restype = C.c_double
        lib.orc_hstar.argtypes = [C.c_double] * 5 + [dp]
        lib.orc_hllc.argtypes = [C.c_double] * 8 + [dp, dp]
        lib.orc_hll.argtypes = [C.c_double] * 8 + [dp]
        lib.orc_mesh_set_flux.argtypes = [vp, C.c_int]
        lib.orc_friction_update.argtypes = [C.c_double] * 10 + [dp]
        lib.orc_step.restype = C.c_int64
        lib.orc_step.argtypes = [vp, dp, dp, dp, C.c_double, dp, dp, dp]
        lib.orc_step_cells.restype = C.c_int64
        lib.orc_step_cells.argtypes = [vp, dp, dp, dp, C.c_double, lp, C.c_int64, dp, dp, dp]
        lib.orc_rhs.argtypes = [vp, dp, dp, dp, dp, dp, dp]
        lib.orc_dt.restype = C.c_double
        lib.orc_dt.argtypes = [vp, dp, dp, dp, C.c_double]
        lib.orc_set_threads.argtypes = [C.c_int]
        lib.orc_max_threads.restype = C.c_int
        lib.orc_run.restype = C.c_int64
        lib.orc_run.argtypes = [vp, dp, dp, dp, C.c_int64, C.c_double, dp, dp]
        lib.orc_run_fixed_dt.restype = C.c_int64
        lib.orc_run_fixed_dt.argtypes = [vp, dp, dp, dp, C.c_int64, dp]
        _lib = lib
        return lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops (timing only; results do not depend on it)."""
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    """Threads the oracle's OpenMP loops use."""
    return int(_load().orc_max_threads())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


class Mesh:
    """The oracle's own mesh: orientation, neighbours and geometry are built
    by the oracle from nodes and triangles alone (Section 3.1, Eq 9, Eq 15)."""

    def __init__(self, nodes, tris, z, m, g=G_DEFAULT, h_dry=H_DRY_DEFAULT):
        lib = _load()
        self.nodes = _f64(nodes).reshape(-1, 2)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
        self.z = _f64(z).reshape(-1).copy()
        self.m = _f64(m).reshape(-1).copy()
        self.g, self.h_dry = float(g), float(h_dry)
        self.n_cells = self.tris.shape[0]
        err = C.c_int(0)
        self._h = lib.orc_mesh_new(_d(self.nodes), self.nodes.shape[0],
                                   self.tris.ctypes.data_as(C.POINTER(C.c_int32)),
                                   self.n_cells, _d(self.z), _d(self.m), self.g, self.h_dry,
                                   C.byref(err))
        if not self._h:
            raise OracleError(f"oracle mesh build failed (code {err.value})")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_mesh_free(h)
            self._h = None

    def set_bc(self, node_pairs, kind, value=0.0) -> int:
        pairs = np.ascontiguousarray(node_pairs, dtype=np.int32).reshape(-1, 2)
        r = _load().orc_mesh_set_bc(self._h, pairs.ctypes.data_as(C.POINTER(C.c_int32)),
                                    pairs.shape[0], int(kind), float(value))
        if r < 0:
            raise OracleError(f"set_bc failed ({-r})")
        return r

    def set_fields(self, z=None, m=None):
        zz = _f64(z) if z is not None else None
        mm = _f64(m) if m is not None else None
        _load().orc_mesh_set_fields(self._h, _d(zz) if zz is not None else None,
                                    _d(mm) if mm is not None else None)
        if zz is not None:
            self.z = zz.copy()
        if mm is not None:
            self.m = mm.copy()

    def geometry(self):
        n = self.n_cells
        area, rin = np.empty(n), np.empty(n)
        nbr = np.empty((n, 3), np.int64)
        ln, nx, ny = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3))
        _load().orc_mesh_geometry(self._h, _d(area), _d(rin),
                                  nbr.ctypes.data_as(C.POINTER(C.c_int64)), _d(ln), _d(nx), _d(ny))
        return dict(area=area, rin=rin, nbr=nbr, len=ln, nx=nx, ny=ny)

    def set_flux(self, hll_only):
        """0: HLLC (default), 1: HLL for all three components."""
        _load().orc_mesh_set_flux(self._h, int(bool(hll_only)))

    def groups(self):
        """Boundary groups as (kind[], value[], total length[]); group 0 is the wall."""
        kind = np.zeros(64, np.int32)
        value, glen = np.zeros(64), np.zeros(64)
        ng = _load().orc_mesh_groups(self._h, kind.ctypes.data_as(C.POINTER(C.c_int)), _d(value), _d(glen))
        return kind[:ng].copy(), value[:ng].copy(), glen[:ng].copy()

    def discharge(self, h, hu, hv):
        """Outward discharge (m^3/s) through each boundary group for this state."""
        h, hu, hv = _f64(h), _f64(hu), _f64(hv)
        Q = np.zeros(64)
        ng = _load().orc_boundary_discharge(self._h, _d(h), _d(hu), _d(hv), _d(Q))
        return Q[:ng].copy()

    def dt(self, h, hu, hv, cfl):
        h, hu, hv = _f64(h), _f64(hu), _f64(hv)
        return _load().orc_dt(self._h, _d(h), _d(hu), _d(hv), float(cfl))

    def rhs(self, h, hu, hv):
        h, hu, hv = _f64(h), _f64(hu), _f64(hv)
        R = [np.empty(self.n_cells) for _ in range(3)]
        _load().orc_rhs(self._h, _d(h), _d(hu), _d(hv), *[_d(r) for r in R])
        return R

    def step(self, h, hu, hv, dt):
        """One explicit Euler step of size dt; returns (h, hu, hv, n_clamped)."""
        h, hu, hv = _f64(h), _f64(hu), _f64(hv)
        out = [np.empty(self.n_cells) for _ in range(3)]
        c = _load().orc_step(self._h, _d(h), _d(hu), _d(hv), float(dt), *[_d(o) for o in out])
        return out[0], out[1], out[2], int(c)

    def step_cells(self, h, hu, hv, dt, cells):
        """One step evaluated only at the listed cells (sampled parity)."""
        h, hu, hv = _f64(h), _f64(hu), _f64(hv)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = [np.empty(cells.shape[0]) for _ in range(3)]
        c = _load().orc_step_cells(self._h, _d(h), _d(hu), _d(hv), float(dt),
                                   cells.ctypes.data_as(C.POINTER(C.c_int64)), cells.shape[0],
                                   *[_d(o) for o in out])
        return out[0], out[1], out[2], int(c)

    def run(self, h, hu, hv, nsteps, cfl, t0=0.0, log_dt=False):
        """nsteps steps with the CFL step recomputed after every update.
        Returns (h, hu, hv, t, n_clamped[, dts])."""
        h, hu, hv = _f64(h).copy(), _f64(hu).copy(), _f64(hv).copy()
        t = C.c_double(t0)
        dts = np.zeros(max(int(nsteps), 1))
        c = _load().orc_run(self._h, _d(h), _d(hu), _d(hv), int(nsteps), float(cfl),
                            C.byref(t), _d(dts))
        if c == -1:
            raise OracleError("every cell is dry: no time step")
        if c < 0:
            raise OracleError("oracle out of memory")
        if log_dt:
            return h, hu, hv, t.value, int(c), dts[: int(nsteps)]
        return h, hu, hv, t.value, int(c)

    def run_fixed_dt(self, h, hu, hv, dts):
        h, hu, hv = _f64(h).copy(), _f64(hu).copy(), _f64(hv).copy()
        dts = _f64(dts)
        c = _load().orc_run_fixed_dt(self._h, _d(h), _d(hu), _d(hv), dts.shape[0], _d(dts))
        return h, hu, hv, int(c)


def hstar(hL, unL, hR, unR, g=G_DEFAULT):
    """Star-region depth estimate of Eq 21-23; returns (h*, h0*)."""
    h0 = C.c_double(0.0)
    hs = _load().orc_hstar(float(hL), float(unL), float(hR), float(unR), float(g), C.byref(h0))
    return hs, h0.value


def hllc(hL, unL, utL, hR, unR, utR, g=G_DEFAULT, h_dry=H_DRY_DEFAULT):
    """HLLC flux (Eq 17-26) in the normal frame; returns (G[3], (S_L, S_R, S*))."""
    G = np.zeros(3)
    S = np.zeros(3)
    _load().orc_hllc(float(hL), float(unL), float(utL), float(hR), float(unR), float(utR),
                     float(g), float(h_dry), _d(G), _d(S))
    return G, S


def hll(hL, unL, utL, hR, unR, utR, g=G_DEFAULT, h_dry=H_DRY_DEFAULT):
    """HLL flux (Eq 17-18) for all three components in the normal frame."""
    G = np.zeros(3)
    _load().orc_hll(float(hL), float(unL), float(utL), float(hR), float(unR), float(utR),
                    float(g), float(h_dry), _d(G))
    return G


def friction_update(h, hu, hv, Rh, Rhu, Rhv, m, dt, g=G_DEFAULT, h_dry=H_DRY_DEFAULT):
    """dU of the semi-implicit step [I - dt/2 J_f] dU = dt (R + S_f) (Eq 33-37)."""
    out = np.zeros(3)
    _load().orc_friction_update(float(h), float(hu), float(hv), float(Rh), float(Rhu), float(Rhv),
                                float(m), float(dt), float(g), float(h_dry), _d(out))
    return out


def rel_err(a, ref):
    """Max relative error per field: max|a - ref| / max(max|ref|, 1e-30)."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(a - ref)) / max(float(np.max(np.abs(ref))), 1e-30)) if ref.size else 0.0
