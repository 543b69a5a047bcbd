"""Diagnostics (stored volume, inflow/outflow rates of Section 5.3.2) and the
run-to-steady-state driver (the stabilised first phase of Section 6.3.2)."""
import numpy as np
import pytest

import oracle
from oracle import rel_err
from paper_2010_14416_gb300 import build as libbuild
from paper_2010_14416_gb300 import capi
from paper_2010_14416_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    libbuild.build()
    return capi.load()


def _pair(mi, precision=capi.SWE_FP64):
    m = capi.Mesh(mi.nodes, mi.tris, mi.z, mi.manning, precision=precision)
    M = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    for pairs, kind, value in mi.bcs:
        m.set_bc(pairs, kind, value)
        M.set_bc(pairs, kind, value)
    d = m.dtype
    m.set_state(mi.h.astype(d), mi.hu.astype(d), mi.hv.astype(d))
    return m, M


@pytest.mark.parametrize("precision,tol", [(capi.SWE_FP64, 1e-12), (capi.SWE_FP32, 1e-5)])
def test_diagnostics_of_seeded_state_against_oracle(precision, tol):
    mi = mg.river(160, 32, seed=5)
    rng = np.random.default_rng(2)
    mi.hu = rng.uniform(-1, 1, mi.n_cells) * mi.h      # moving water at the stage edge
    mi.hv = rng.uniform(-1, 1, mi.n_cells) * mi.h
    m, M = _pair(mi, precision)
    d = m.diagnostics()
    area = M.geometry()["area"]
    u0 = [a.astype(m.dtype).astype(np.float64) for a in (mi.h, mi.hu, mi.hv)]
    Q = M.discharge(*u0)
    assert d["n_groups"] == 3 and d["dt_last"] == 0.0
    assert d["volume"] == pytest.approx((area * u0[0]).sum(), rel=tol)
    assert rel_err(d["discharge"], Q) <= tol
    assert d["discharge"][1] == pytest.approx(-mi.meta["Q"], rel=tol)
    assert d["h_max"] == pytest.approx(u0[0].max(), rel=1e-15)
    assert d["n_wet"] == int((u0[0] > 1e-6).sum())
    m.close()


def test_volume_balance_identity_over_steps():
    # interior fluxes cancel: V^{n+1} - V^n = -dt_n * sum_g Q_g(U^n)
    mi = mg.river(160, 32, seed=6, Q=800.0)
    m, _ = _pair(mi)
    prev = m.diagnostics()
    for _ in range(40):
        m.step(1)
        d = m.diagnostics()
        dv = d["volume"] - prev["volume"]
        assert dv == pytest.approx(-d["dt_last"] * prev["discharge"].sum(), rel=1e-9, abs=1e-12 * d["volume"])
        prev = d
    m.close()


def test_run_to_steady_state_balances_inflow_and_outflow():
    # a short sloping canal: inflow upstream, fixed stage downstream
    mi = mg.canal(60, 6, 300.0, 30.0, 0.2, 4, hL=1.0, hR=1.0, manning=0.03)
    mi.z = 1e-3 * (300.0 - mi.centroids()[:, 0])
    mi.h = np.maximum(1.0 - mi.z, 0.0)
    sides = mg._side_pairs(60, 6)
    mi.bcs = [(sides["left"].astype(np.int32), mg.BC_INFLOW, 30.0),
              (sides["right"].astype(np.int32), mg.BC_STAGE, 1.0)]
    m, _ = _pair(mi)
    steps, conv, t = m.run_to_steady(tol=1e-7, check_every=500, max_steps=200000)
    assert conv and steps < 200000
    d = m.diagnostics()
    q_in, q_out = -d["discharge"][1], d["discharge"][2]
    assert q_in == pytest.approx(30.0, rel=1e-12)
    assert q_out == pytest.approx(q_in, rel=1e-3)
    m.close()
