"""The allocation-free CFL step, swe_cfl_dt_noalloc.

It serves callers that cannot let the library allocate device memory (an
own memory arena, or a CUDA graph being captured).  Its answer must equal the
first time step that the allocating path (swe_set_state) computes for the
same state, call after call, although all calls share one static scratch
array.  This file is collected last so that a failure here comes after every
other test has run."""
import ctypes as C

import numpy as np
import pytest

from paper_2010_14416_gb300 import build as libbuild
from paper_2010_14416_gb300 import capi
from paper_2010_14416_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {capi.SWE_FP64: 1e-10, capi.SWE_FP32: 1e-4}
CFL = 0.9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    libbuild.build()
    return capi.load()


def _allocating_dt(mi, precision, state):
    """CFL step of `state` as computed by the allocating path."""
    m = capi.Mesh(mi.nodes, mi.tris, mi.z, mi.manning, precision=precision)
    npdt = np.float32 if precision == capi.SWE_FP32 else np.float64
    m.set_state(*(a.astype(npdt) for a in state))
    raw = m.info()["dt_next"]
    m.close()
    return CFL * raw


@pytest.mark.parametrize("precision", [capi.SWE_FP64, capi.SWE_FP32])
def test_noalloc_dt_matches_allocating_path_twice(precision):
    mi = mg.river(200, 40, seed=11)          # partially dry, 16,000 cells
    pre = capi.mesh_preprocess(mi.nodes, mi.tris)
    rin = np.empty(mi.n_cells)
    rin[pre["perm"]] = pre["rin"]            # caller order
    tdt = torch.float32 if precision == capi.SWE_FP32 else torch.float64
    rng = np.random.default_rng(5)
    state_a = (mi.h, mi.hu, mi.hv)
    hb = mi.h * rng.uniform(0.5, 1.5, mi.n_cells)
    state_b = (hb, rng.uniform(-2, 2, mi.n_cells) * hb, rng.uniform(-2, 2, mi.n_cells) * hb)
    d_rin = torch.tensor(rin, dtype=tdt, device="cuda")
    dt_out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    for state in (state_a, state_b):         # two calls in a row, different states
        dev = [torch.tensor(a, dtype=tdt, device="cuda") for a in state]
        capi.cfl_dt_noalloc(precision, *dev, d_rin, dt_out, cfl=CFL)
        torch.cuda.synchronize()
        got = float(dt_out.item())
        ref = _allocating_dt(mi, precision, state)
        assert np.isfinite(ref) and ref > 0
        assert abs(got - ref) <= TOL[precision] * ref, (got, ref)


def test_noalloc_all_dry_and_size_limit():
    n = 1000
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    rin = torch.ones(n, dtype=torch.float64, device="cuda")
    dt_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    capi.cfl_dt_noalloc(capi.SWE_FP64, z, z, z, rin, dt_out)
    torch.cuda.synchronize()
    assert dt_out.item() == float("inf")
    # beyond the stated maximum the call is refused before touching memory
    lib = capi.load()
    p = C.c_void_p(z.data_ptr())
    rc = lib.swe_cfl_dt_noalloc(capi.SWE_FP64, 16_777_217, p, p, p, p, 9.81, 1e-6, 0.9,
                                C.c_void_p(dt_out.data_ptr()), None)
    assert rc == capi.SWE_EINVAL
    assert b"allocation-free limit" in lib.swe_last_error()
