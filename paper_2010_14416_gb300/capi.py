"""ctypes binding of libswe's C ABI (include/swe.h), with the same names.

Argument marshalling only: every step of the solver runs in the CUDA library.
Arrays may be numpy arrays (host) or torch tensors (host or CUDA); CUDA
tensors are passed as device pointers and the mesh runs on torch's current
stream unless another stream is set.  The library must have been built
(``paper_2010_14416_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libswe.so")

SWE_OK, SWE_EINVAL, SWE_EMESH, SWE_ENOMEM, SWE_ECUDA, SWE_ENONFINITE, SWE_EDRY, SWE_ETIMEOUT = range(8)
SWE_FP64, SWE_FP32 = 0, 1
SWE_REORDER_NONE, SWE_REORDER_RCM, SWE_REORDER_HILBERT = 0, 1, 2
SWE_BC_WALL, SWE_BC_INFLOW, SWE_BC_TRANSMISSIVE, SWE_BC_STAGE = 0, 1, 2, 3
SWE_HOST, SWE_DEVICE = 0, 1
SWE_FLUX_HLLC, SWE_FLUX_HLL = 0, 1
SWE_ADJOINT_TRANSPOSE, SWE_ADJOINT_DUAL = 0, 1

ERROR_NAMES = {1: "SWE_EINVAL", 2: "SWE_EMESH", 3: "SWE_ENOMEM", 4: "SWE_ECUDA",
               5: "SWE_ENONFINITE", 6: "SWE_EDRY", 7: "SWE_ETIMEOUT"}

# every symbol include/swe.h declares
EXPORTS = ["swe_config_default", "swe_mesh_create", "swe_mesh_destroy", "swe_set_bc",
           "swe_set_stream", "swe_set_state", "swe_step", "swe_get_state", "swe_synchronize",
           "swe_get_info", "swe_get_permutation", "swe_mesh_preprocess", "swe_riemann_flux", "swe_riemann_flux_kind",
           "swe_cfl_dt_noalloc", "swe_ensemble_create", "swe_ensemble_destroy", "swe_ensemble_set_stream",
           "swe_ensemble_step", "swe_ensemble_get_state", "swe_ensemble_get_info", "swe_adjoint",
           "swe_adjoint_series",
           "swe_step_dt", "swe_set_fields", "swe_diagnostics", "swe_run_to_steady", "swe_autotune",
           "swe_ensemble_autotune", "swe_ensemble_set_shape", "swe_debug_code_ok", "swe_adjoint_method",
           "swe_last_error"]


class swe_config(C.Structure):
    _fields_ = [("precision", C.c_int), ("g", C.c_double), ("h_dry", C.c_double),
                ("reorder", C.c_int), ("block_size", C.c_int), ("graph_steps", C.c_int),
                ("device", C.c_int), ("min_blocks", C.c_int), ("stages", C.c_int), ("flux", C.c_int),
                ("geometry_early", C.c_int), ("activity", C.c_int), ("edge_pass", C.c_int), ("grid", C.c_int),
                ("debug_checks", C.c_int), ("cell_pairs", C.c_int)]


class swe_info(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("n_steps", C.c_int64), ("n_clamped", C.c_int64),
                ("t", C.c_double), ("dt_next", C.c_double), ("precision", C.c_int),
                ("status", C.c_int), ("device_bytes", C.c_int64), ("n_active", C.c_int64)]


class swe_diag(C.Structure):
    _fields_ = [("t", C.c_double), ("dt_last", C.c_double), ("volume", C.c_double), ("dh_max", C.c_double),
                ("h_max", C.c_double), ("speed_max", C.c_double), ("n_wet", C.c_int64), ("n_groups", C.c_int),
                ("discharge", C.c_double * 64)]


class swe_tune(C.Structure):
    _fields_ = [("block_size", C.c_int), ("min_blocks", C.c_int), ("stages", C.c_int), ("geometry_early", C.c_int),
                ("activity", C.c_int), ("edge_pass", C.c_int), ("dynamic", C.c_int), ("chunk", C.c_int),
                ("grid", C.c_int64), ("cells_per_thread", C.c_double), ("ms_best", C.c_double),
                ("ms_before", C.c_double), ("n_candidates", C.c_int), ("cell_pairs", C.c_int), ("queue", C.c_int)]


class SWEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load():
    """Loads libswe.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libswe.so is not built ({LIB_PATH}); run "
                           "paper_2010_14416_gb300.build.build() -- there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    vp, dp = C.c_void_p, C.POINTER(C.c_double)
    lib.swe_config_default.argtypes = [C.POINTER(swe_config)]
    lib.swe_config_default.restype = None
    lib.swe_mesh_create.argtypes = [vp, C.c_int64, vp, C.c_int64, vp, vp, C.POINTER(swe_config),
                                    C.POINTER(vp)]
    lib.swe_mesh_destroy.argtypes = [vp]
    lib.swe_mesh_destroy.restype = None
    lib.swe_set_bc.argtypes = [vp, vp, C.c_int64, C.c_int, C.c_double]
    lib.swe_set_stream.argtypes = [vp, vp]
    lib.swe_set_state.argtypes = [vp, vp, vp, vp, C.c_int, C.c_double]
    lib.swe_step.argtypes = [vp, C.c_int64, C.c_double, dp]
    lib.swe_get_state.argtypes = [vp, vp, vp, vp, C.c_int]
    lib.swe_synchronize.argtypes = [vp]
    lib.swe_get_info.argtypes = [vp, C.POINTER(swe_info)]
    lib.swe_get_permutation.argtypes = [vp, vp]
    lib.swe_riemann_flux.argtypes = [C.c_int, C.c_int64] + [vp] * 6 + [C.c_double, C.c_double] + \
        [vp] * 4 + [vp]
    lib.swe_riemann_flux_kind.argtypes = [C.c_int, C.c_int, C.c_int64] + [vp] * 6 + [C.c_double, C.c_double] + \
        [vp] * 4 + [vp]
    lib.swe_mesh_preprocess.argtypes = [vp, C.c_int64, vp, C.c_int64, C.c_int, C.c_int, vp, vp, vp, vp, vp]
    lib.swe_debug_code_ok.argtypes = [C.c_int32, C.c_int64, C.c_int]
    lib.swe_cfl_dt_noalloc.argtypes = [C.c_int, C.c_int64, vp, vp, vp, vp, C.c_double, C.c_double,
                                       C.c_double, vp, vp]
    lib.swe_ensemble_create.argtypes = [vp, C.c_int, C.POINTER(vp)]
    lib.swe_ensemble_destroy.argtypes = [vp]
    lib.swe_ensemble_destroy.restype = None
    lib.swe_ensemble_set_stream.argtypes = [vp, vp]
    lib.swe_ensemble_step.argtypes = [vp, C.c_int64, vp, vp]
    lib.swe_ensemble_get_state.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int]
    lib.swe_ensemble_get_info.argtypes = [vp, C.c_int, C.POINTER(swe_info)]
    lib.swe_adjoint.argtypes = [vp, C.c_int64, C.c_double, vp, C.c_int, vp, C.c_int, vp, vp, vp, C.c_int, vp]
    lib.swe_adjoint_series.argtypes = [vp, C.c_int64, C.c_double, vp, C.c_int, vp, C.c_int64, C.c_int, vp, vp,
                                       vp, C.c_int, vp]
    lib.swe_step_dt.argtypes = [vp, C.c_int64, vp, vp]
    lib.swe_set_fields.argtypes = [vp, vp, vp]
    lib.swe_diagnostics.argtypes = [vp, C.POINTER(swe_diag)]
    lib.swe_run_to_steady.argtypes = [vp, C.c_double, C.c_double, C.c_int64, C.c_int64, C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int), C.POINTER(C.c_double)]
    lib.swe_autotune.argtypes = [vp, C.c_int, C.POINTER(swe_tune)]
    lib.swe_ensemble_autotune.argtypes = [vp, C.c_int, C.POINTER(swe_tune)]
    lib.swe_ensemble_set_shape.argtypes = [vp, C.POINTER(swe_tune)]
    lib.swe_last_error.argtypes = []
    lib.swe_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("swe_config_default", "swe_mesh_destroy", "swe_ensemble_destroy", "swe_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def check(rc):
    if rc != SWE_OK:
        raise SWEError(rc, load().swe_last_error().decode())
    return rc


def _ptr(a, dtype=None):
    """(pointer, where, keepalive) for a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if dtype is not None:
                want = {np.float64: torch.float64, np.float32: torch.float32}[np.dtype(dtype).type]
                if a.dtype != want:
                    raise TypeError(f"expected {want}, got {a.dtype}")
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return a.data_ptr(), (SWE_DEVICE if a.is_cuda else SWE_HOST), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype) if dtype is not None else np.ascontiguousarray(a)
    return arr.ctypes.data, SWE_HOST, arr


def config_default():
    cfg = swe_config()
    load().swe_config_default(C.byref(cfg))
    return cfg


class Mesh:
    """An owned swe_mesh handle (thin wrapper over the C ABI)."""

    def __init__(self, nodes, tris, bathy, manning, precision=SWE_FP64, reorder=None,
                 block_size=0, graph_steps=0, device=0, g=9.81, h_dry=1e-6, min_blocks=0, stages=0,
                 flux=SWE_FLUX_HLLC, geometry_early=0, activity=0, edge_pass=0, grid=0, debug_checks=0,
                 cell_pairs=0):
        lib = load()
        cfg = config_default()
        cfg.precision = precision
        if reorder is not None:
            cfg.reorder = reorder
        cfg.block_size, cfg.graph_steps, cfg.device = block_size, graph_steps, device
        cfg.min_blocks = min_blocks
        cfg.stages = stages
        cfg.geometry_early = geometry_early
        cfg.activity = activity
        cfg.edge_pass = edge_pass
        cfg.grid = grid
        cfg.debug_checks = debug_checks
        cfg.cell_pairs = cell_pairs
        cfg.flux = flux
        cfg.g, cfg.h_dry = g, h_dry
        nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(-1, 2)
        tris = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
        bathy = np.ascontiguousarray(bathy, dtype=np.float64).reshape(-1)
        manning = np.ascontiguousarray(manning, dtype=np.float64).reshape(-1)
        if bathy.shape[0] != tris.shape[0] or manning.shape[0] != tris.shape[0]:
            raise ValueError("bathy and manning need one value per triangle")
        h = C.c_void_p()
        check(lib.swe_mesh_create(nodes.ctypes.data, nodes.shape[0], tris.ctypes.data, tris.shape[0],
                                  bathy.ctypes.data, manning.ctypes.data, C.byref(cfg), C.byref(h)))
        self._h = h
        self.n_cells = tris.shape[0]
        self.precision = precision
        self.dtype = np.float32 if precision == SWE_FP32 else np.float64
        self.device = device
        self._stream = None

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.swe_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def set_bc(self, node_pairs, kind, value=0.0):
        p = np.ascontiguousarray(node_pairs, dtype=np.int32).reshape(-1, 2)
        check(load().swe_set_bc(self._h, p.ctypes.data, p.shape[0], int(kind), float(value)))

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        self._stream = raw
        check(load().swe_set_stream(self._h, C.c_void_p(raw or 0)))

    def _use_torch_stream(self, where):
        if where == SWE_DEVICE and self._stream is None:
            import torch
            check(load().swe_set_stream(self._h, C.c_void_p(torch.cuda.current_stream().cuda_stream)))

    def set_state(self, h, hu, hv, t=0.0):
        ph, w0, k0 = _ptr(h, self.dtype)
        pu, w1, k1 = _ptr(hu, self.dtype)
        pv, w2, k2 = _ptr(hv, self.dtype)
        if not (w0 == w1 == w2):
            raise ValueError("h, hu, hv must all be on the host or all on the device")
        self._use_torch_stream(w0)
        check(load().swe_set_state(self._h, ph, pu, pv, w0, float(t)))

    def step(self, nsteps, cfl=0.9, sync=True):
        """Advances nsteps; returns the time reached when sync is true."""
        t = C.c_double(0.0)
        check(load().swe_step(self._h, int(nsteps), float(cfl), C.byref(t) if sync else None))
        return t.value if sync else None

    def get_state(self, out=None):
        """Returns (h, hu, hv); host numpy arrays unless `out` gives buffers."""
        if out is None:
            out = tuple(np.empty(self.n_cells, self.dtype) for _ in range(3))
        ptrs = [_ptr(o, self.dtype) for o in out]
        where = ptrs[0][1]
        self._use_torch_stream(where)
        check(load().swe_get_state(self._h, ptrs[0][0], ptrs[1][0], ptrs[2][0], where))
        return out

    def synchronize(self):
        check(load().swe_synchronize(self._h))

    def info(self):
        inf = swe_info()
        check(load().swe_get_info(self._h, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in swe_info._fields_}

    def adjoint_method(self, method):
        """SWE_ADJOINT_TRANSPOSE (default) or SWE_ADJOINT_DUAL: how the reverse
        step forms its edge terms (see swe_adjoint_method)."""
        check(load().swe_adjoint_method(self._h, int(method)))

    def adjoint(self, nsteps, gauges, target, cfl=0.9, checkpoint_every=50, out=None):
        """Gauge-misfit loss after nsteps and its gradient w.r.t. (manning,
        bathy); returns (loss, grad_manning, grad_bathy, dts).  `out` may give
        two device tensors for the gradients."""
        g = np.ascontiguousarray(gauges, dtype=np.int32)
        t = np.ascontiguousarray(target, dtype=np.float64)
        loss = C.c_double(0.0)
        dts = np.zeros(int(nsteps))
        if out is None:
            gm, gz = np.zeros(self.n_cells), np.zeros(self.n_cells)
            pm, pz, where = gm.ctypes.data, gz.ctypes.data, SWE_HOST
        else:
            gm, gz = out
            pm, pz, where = gm.data_ptr(), gz.data_ptr(), SWE_DEVICE
        check(load().swe_adjoint(self._h, int(nsteps), float(cfl), g.ctypes.data, g.shape[0], t.ctypes.data,
                                 int(checkpoint_every), C.byref(loss), pm, pz, where, dts.ctypes.data))
        return loss.value, gm, gz, dts

    def adjoint_series(self, nsteps, gauges, targets, obs_every, cfl=0.9, checkpoint_every=50):
        """Time-series misfit over observations every obs_every steps and its
        gradient; targets: [nsteps // obs_every, n_gauges].  Returns
        (loss, grad_manning, grad_bathy, dts)."""
        g = np.ascontiguousarray(gauges, dtype=np.int32)
        t = np.ascontiguousarray(targets, dtype=np.float64)
        loss = C.c_double(0.0)
        dts = np.zeros(int(nsteps))
        gm, gz = np.zeros(self.n_cells), np.zeros(self.n_cells)
        check(load().swe_adjoint_series(self._h, int(nsteps), float(cfl), g.ctypes.data, g.shape[0], t.ctypes.data,
                                        int(obs_every), int(checkpoint_every), C.byref(loss), gm.ctypes.data,
                                        gz.ctypes.data, SWE_HOST, dts.ctypes.data))
        return loss.value, gm, gz, dts

    def step_dt(self, dts):
        d = np.ascontiguousarray(dts, dtype=np.float64)
        t = C.c_double(0.0)
        check(load().swe_step_dt(self._h, d.shape[0], d.ctypes.data, C.byref(t)))
        return t.value

    def set_fields(self, bathy=None, manning=None):
        b = np.ascontiguousarray(bathy, dtype=np.float64) if bathy is not None else None
        mm = np.ascontiguousarray(manning, dtype=np.float64) if manning is not None else None
        check(load().swe_set_fields(self._h, b.ctypes.data if b is not None else None,
                                    mm.ctypes.data if mm is not None else None))

    def diagnostics(self):
        """Volume, last-step depth change, extremes, wet cells and the outward
        discharge of each boundary group (group 0 = default wall)."""
        d = swe_diag()
        check(load().swe_diagnostics(self._h, C.byref(d)))
        out = {k: getattr(d, k) for k, _ in swe_diag._fields_ if k != "discharge"}
        out["discharge"] = np.array(d.discharge[: d.n_groups])
        return out

    def run_to_steady(self, tol, cfl=0.9, check_every=100, max_steps=100000):
        """Steps until max |dh|/dt < tol; returns (steps, converged, t)."""
        n = C.c_int64(0)
        conv = C.c_int(0)
        t = C.c_double(0.0)
        check(load().swe_run_to_steady(self._h, float(cfl), float(tol), int(check_every), int(max_steps),
                                       C.byref(n), C.byref(conv), C.byref(t)))
        return n.value, bool(conv.value), t.value

    def autotune(self, trial_steps=8):
        """Times the step kernel's compiled launch shapes on the current state
        (which does not change) and keeps the fastest; returns the choice."""
        t = swe_tune()
        check(load().swe_autotune(self._h, int(trial_steps), C.byref(t)))
        return {k: getattr(t, k) for k, _ in swe_tune._fields_}

    def permutation(self):
        p = np.empty(self.n_cells, np.int64)
        check(load().swe_get_permutation(self._h, p.ctypes.data))
        return p


class Ensemble:
    """Members advanced together in one CUDA-graph launch per call."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        arr = (C.c_void_p * len(self.meshes))(*[m.handle.value for m in self.meshes])
        h = C.c_void_p()
        check(load().swe_ensemble_create(arr, len(self.meshes), C.byref(h)))
        self._h = h
        self.n_members = len(self.meshes)
        self.dtype = self.meshes[0].dtype

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.swe_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def set_stream(self, stream):
        raw = getattr(stream, "cuda_stream", stream)
        check(load().swe_ensemble_set_stream(self._h, C.c_void_p(raw or 0)))

    def step(self, nsteps, cfl=None, sync=True):
        c = None
        if cfl is not None:
            c = np.ascontiguousarray(np.broadcast_to(np.asarray(cfl, np.float64), (self.n_members,)))
        t = np.zeros(self.n_members) if sync else None
        check(load().swe_ensemble_step(self._h, int(nsteps), c.ctypes.data if c is not None else None,
                                       t.ctypes.data if sync else None))
        return t

    def get_state(self, member, out=None):
        n = self.meshes[member].n_cells
        if out is None:
            out = tuple(np.empty(n, self.dtype) for _ in range(3))
        ptrs = [_ptr(o, self.dtype) for o in out]
        check(load().swe_ensemble_get_state(self._h, int(member), ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[0][1]))
        return out

    def autotune(self, trial_steps=4):
        """Times the batched kernel's launch shapes (tile size, staging, chunk,
        grid) on the current states and keeps the fastest; returns the choice."""
        t = swe_tune()
        check(load().swe_ensemble_autotune(self._h, int(trial_steps), C.byref(t)))
        return {k: getattr(t, k) for k, _ in swe_tune._fields_}

    def set_shape(self, block_size, min_blocks, stages=1, geometry_early=0, activity=0, chunk=4, grid=0,
                  edge_pass=0, dynamic=0, cell_pairs=0, queue=0):
        """Sets the batched kernel's launch shape (see swe_ensemble_set_shape);
        cell_pairs=1: the split step, queue=1: per-warp queues (FP32)."""
        t = swe_tune(block_size=block_size, min_blocks=min_blocks, stages=stages, geometry_early=geometry_early,
                     activity=activity, edge_pass=edge_pass, dynamic=dynamic, chunk=chunk, grid=grid,
                     cell_pairs=cell_pairs, queue=queue)
        check(load().swe_ensemble_set_shape(self._h, C.byref(t)))

    def info(self, member):
        inf = swe_info()
        check(load().swe_ensemble_get_info(self._h, int(member), C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in swe_info._fields_}


def mesh_preprocess(nodes, tris, reorder=SWE_REORDER_HILBERT, precision=SWE_FP64):
    """Host-only preprocessing (no GPU) of a mesh of the given precision: perm,
    code, ln, inv_area, rin in internal order."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(-1, 2)
    tris = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
    n = tris.shape[0]
    perm = np.empty(n, np.int64)
    code = np.empty((n, 3), np.int32)
    ln = np.empty((n, 3, 2))
    ia = np.empty(n)
    rin = np.empty(n)
    check(load().swe_mesh_preprocess(nodes.ctypes.data, nodes.shape[0], tris.ctypes.data, n, int(reorder),
                                     int(precision), perm.ctypes.data, code.ctypes.data, ln.ctypes.data, ia.ctypes.data,
                                     rin.ctypes.data))
    return dict(perm=perm, code=code, ln=ln, inv_area=ia, rin=rin)


def debug_code_ok(code, n_cells, n_groups):
    """swe_debug_code_ok: whether a neighbour code is usable on a mesh of
    n_cells cells with n_groups boundary groups (the debug-checks predicate)."""
    return bool(load().swe_debug_code_ok(int(np.int32(code)), int(n_cells), int(n_groups)))


def riemann_flux(precision, hL, unL, utL, hR, unR, utR, G1, G2, G3, S=None, g=9.81, h_dry=1e-6,
                 stream=None, flux=SWE_FLUX_HLLC):
    """Batched normal-frame Riemann flux on device tensors (parity entry)."""
    n = hL.numel()
    ptrs = [t.data_ptr() for t in (hL, unL, utL, hR, unR, utR)]
    outs = [t.data_ptr() for t in (G1, G2, G3)]
    sp = S.data_ptr() if S is not None else None
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    check(load().swe_riemann_flux_kind(precision, flux, n, *ptrs, g, h_dry, *outs, sp, C.c_void_p(stream)))


def cfl_dt_noalloc(precision, h, hu, hv, rin, dt_out, cfl=0.9, g=9.81, h_dry=1e-6, stream=None):
    """Allocation-free CFL step of a state held in device tensors; writes
    cfl * min R/(c+|u|) into the one-element device tensor dt_out."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    check(load().swe_cfl_dt_noalloc(precision, h.numel(), h.data_ptr(), hu.data_ptr(), hv.data_ptr(),
                                    rin.data_ptr(), g, h_dry, cfl, dt_out.data_ptr(), C.c_void_p(stream)))
