"""Pins for the oracle's whole step (Eq 16, 27-37, Section 3.1 boundary
conditions, Eq 15 CFL) against invariants, closed forms, analytic dam-break
solutions and brute-force symmetries."""
import math

import numpy as np
import pytest

import oracle
from oracle import analytic
from paper_2010_14416_gb300 import meshgen as mg

G = 9.81


def _mesh(mi, with_bcs=True):
    M = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    if with_bcs:
        for pairs, kind, value in mi.bcs:
            M.set_bc(pairs, kind, value)
    return M


def _run_to(M, h, hu, hv, T, cfl=0.9):
    t = 0.0
    while t < T - 1e-12:
        dt = min(M.dt(h, hu, hv, cfl), T - t)
        h, hu, hv, c = M.step(h, hu, hv, dt)
        assert c == 0
        t += dt
    return h, hu, hv


@pytest.mark.parametrize("fully_wet", [True, False])
def test_lake_at_rest_is_preserved(fully_wet):
    # hydrostatic reconstruction with the 1/2 factor of Eq 30 balances the
    # pressure flux of U** exactly: a flat free surface stays at rest,
    # including around emerged bumps (fully_wet=False leaves dry floodplain)
    mi = mg.river(120, 24, seed=2, fully_wet=fully_wet)
    eta0 = mi.meta["eta0"]
    M = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    M.set_bc(mi.bcs[1][0], oracle.BC_STAGE, eta0)  # no inflow: stage at eta0
    h0 = np.maximum(eta0 - mi.z, 0.0)
    dry = h0 <= 0.0
    if not fully_wet:
        assert dry.sum() > 100
    h, hu, hv, t, c = M.run(h0, np.zeros_like(h0), np.zeros_like(h0), 1000, 0.9)
    assert c == 0
    assert np.abs(h + mi.z - eta0)[~dry].max() < 1e-12
    assert np.all(h[dry] == 0.0)
    assert np.abs(hu).max() < 1e-10 and np.abs(hv).max() < 1e-10


def test_mass_conserved_with_walls():
    mi = mg.dam_break_4k()
    M = _mesh(mi)
    area = M.geometry()["area"]
    m0 = (area * mi.h).sum()
    h, hu, hv, t, c = M.run(mi.h, mi.hu, mi.hv, 500, 0.9)
    assert c == 0
    assert abs((area * h).sum() - m0) / m0 < 500 * 1e-15


def test_inflow_mass_balance():
    # walls everywhere except an inflow of Q on the upstream edges: the
    # stored volume grows by exactly Q t (Section 3.1: G~_1 = -q inward)
    mi = mg.canal(60, 6, 60.0, 6.0, 0.2, 4, hL=1.0, hR=1.0)
    sides = mg._side_pairs(60, 6)
    Q = 3.0
    M = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    M.set_bc(sides["left"].astype(np.int32), oracle.BC_INFLOW, Q)
    area = M.geometry()["area"]
    m0 = (area * mi.h).sum()
    h, hu, hv, t, c = M.run(mi.h, mi.hu, mi.hv, 300, 0.9)
    assert c == 0
    assert ((area * h).sum() - m0) == pytest.approx(Q * t, rel=1e-11)


def test_stage_boundary_at_rest():
    mi = mg.canal(40, 4, 40.0, 4.0, 0.2, 2, hL=2.0, hR=2.0)
    sides = mg._side_pairs(40, 4)
    M = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    M.set_bc(sides["right"].astype(np.int32), oracle.BC_STAGE, 2.0)
    h, hu, hv, t, c = M.run(mi.h, mi.hu, mi.hv, 300, 0.9)
    assert np.abs(h - 2.0).max() < 1e-12 and np.abs(hu).max() < 1e-11
    # a lower stage drains the canal through that edge only
    M2 = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    M2.set_bc(sides["right"].astype(np.int32), oracle.BC_STAGE, 1.0)
    area = M2.geometry()["area"]
    h2, hu2, hv2, t2, c2 = M2.run(mi.h, mi.hu, mi.hv, 100, 0.9)
    assert (area * h2).sum() < (area * mi.h).sum()
    assert hu2.max() > 0.1


def test_transmissive_uniform_flow_is_steady():
    mi = mg.canal(30, 6, 30.0, 6.0, 0.2, 3, side_bc=mg.BC_TRANSMISSIVE, hL=2.0, hR=2.0)
    M = _mesh(mi)
    n = mi.n_cells
    h0, hu0, hv0 = np.full(n, 2.0), np.full(n, 1.4), np.full(n, -0.6)
    h, hu, hv, t, c = M.run(h0, hu0, hv0, 200, 0.9)
    assert np.abs(h - 2.0).max() < 1e-12
    assert np.abs(hu - 1.4).max() < 1e-12 and np.abs(hv + 0.6).max() < 1e-12


def test_friction_uniform_state_closed_form():
    # uniform flow over a flat bed with transmissive edges: R = 0 and q is an
    # eigenvector of J_qq with eigenvalue -2 c |q|, so one step of Eq 37 gives
    # q' = q / (1 + dt c |q|) with c = g m^2 h^{-7/3}, h unchanged
    m = 0.04
    mi = mg.canal(30, 6, 30.0, 6.0, 0.2, 3, side_bc=mg.BC_TRANSMISSIVE, hL=1.5, hR=1.5,
                  manning=m)
    M = _mesh(mi)
    n = mi.n_cells
    h0, hu0, hv0 = np.full(n, 1.5), np.full(n, 3.0), np.full(n, 4.0)
    dt = 0.05
    h, hu, hv, c = M.step(h0, hu0, hv0, dt)
    cc = G * m * m * 1.5 ** (-7.0 / 3.0)
    fac = 1.0 / (1.0 + dt * cc * 5.0)
    assert np.abs(h - 1.5).max() < 1e-13
    assert np.abs(hu - 3.0 * fac).max() < 1e-12
    assert np.abs(hv - 4.0 * fac).max() < 1e-12
    # for dq/dt = -c |q| q the step gives 1/|q'| = 1/|q| + c dt, so any
    # sequence of steps lands exactly on the ODE solution q0 / (1 + c |q0| T)
    rng = np.random.default_rng(5)
    dt_cfl = M.dt(h0, hu0, hv0, 0.9)
    dts = rng.uniform(0.2, 1.0, 200) * dt_cfl
    T = dts.sum()
    h, hu, hv, _ = M.run_fixed_dt(h0, hu0, hv0, dts)
    qex = 5.0 / (1.0 + cc * 5.0 * T)
    assert np.abs(np.hypot(hu, hv) - qex).max() < 1e-12
    assert np.abs(hu * 4.0 - hv * 3.0).max() < 1e-12   # direction kept


def test_friction_update_matches_fd_jacobian_solve():
    # J_f of Eq 35 by central differences of S_f (Eq 32), then the 3x3
    # system [I - dt/2 J] dU = dt (R + S_f) solved by numpy
    rng = np.random.default_rng(11)

    def Sf(U, m):
        h, hu, hv = U
        q = math.hypot(hu, hv)
        c = G * m * m / h ** (7.0 / 3.0)
        return np.array([0.0, -c * q * hu, -c * q * hv])

    for _ in range(50):
        U = np.array([rng.uniform(0.05, 5), rng.uniform(-4, 4), rng.uniform(-4, 4)])
        R = rng.uniform(-2, 2, 3)
        m, dt = rng.uniform(0.01, 0.08), rng.uniform(0.001, 0.5)
        J = np.zeros((3, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6 * max(abs(U[k]), 1e-3)
            J[:, k] = (Sf(U + e, m) - Sf(U - e, m)) / (2 * e[k])
        ref = np.linalg.solve(np.eye(3) - 0.5 * dt * J, dt * (R + Sf(U, m)))
        got = oracle.friction_update(*U, *R, m, dt)
        assert np.allclose(got, ref, rtol=1e-7, atol=1e-9 * (1 + np.abs(ref).max()))


def test_cfl_brute_force_and_closed_form():
    mi = mg.river(50, 10, seed=6)
    M = _mesh(mi)
    geo = M.geometry()
    rng = np.random.default_rng(2)
    n = mi.n_cells
    h = np.where(rng.random(n) < 0.3, 0.0, rng.uniform(0.1, 5, n))
    hu, hv = rng.uniform(-3, 3, n) * h, rng.uniform(-3, 3, n) * h
    brute = min(geo["rin"][i] / (math.sqrt(G * h[i]) + math.hypot(hu[i] / h[i], hv[i] / h[i]))
                for i in range(n) if h[i] > 1e-6)
    assert M.dt(h, hu, hv, 0.9) == pytest.approx(0.9 * brute, rel=1e-15)
    # uniform state: CFL * r_min / (sqrt(g h) + |u|)
    hh = np.full(n, 2.0)
    uu = np.full(n, 2.0 * 1.5)
    vv = np.full(n, 2.0 * -2.0)
    assert M.dt(hh, uu, vv, 0.9) == pytest.approx(
        0.9 * geo["rin"].min() / (math.sqrt(G * 2.0) + 2.5), rel=1e-14)
    assert math.isinf(M.dt(np.zeros(n), np.zeros(n), np.zeros(n), 0.9))


@pytest.mark.parametrize("hR", [1.0, 0.0])
def test_dam_break_converges_to_exact_solution(hR):
    # Stoker (wet bed) and Ritter (dry bed) dam breaks, Section 6.3 oriented
    # along x: the L1 depth error against the exact solution falls with the
    # mesh size (first-order scheme on jittered triangles)
    T = 2.5
    errs = []
    for nx in (100, 200, 400, 800):
        ny = nx // 20
        mi = mg.canal(nx, ny, 200.0, 10.0, 0.2, 1, 10.0, hR, 100.0, 0.0)
        M = _mesh(mi)
        h, hu, hv = _run_to(M, mi.h, mi.hu, mi.hv, T)
        area = M.geometry()["area"]
        cx = mi.centroids()[:, 0]
        he, ue = analytic.dam_break(cx, T, 10.0, hR, 100.0)
        errs.append(np.sum(np.abs(h - he) * area) / area.sum())
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(orders > 0.45), orders
    assert orders.mean() > 0.6, orders
    assert errs[-1] < 0.025


def _mirror_case():
    mi = mg.river(24, 6, Lx=240.0, Ly=60.0, seed=9, Q=40.0, eta0=1.0, stage=1.5,
                  n_bumps=6, shuffle=True)
    rng = np.random.default_rng(1)
    n = mi.n_cells
    h0 = mi.h + rng.uniform(0, 0.3, n) * (mi.h > 0)
    hu0 = rng.uniform(-0.5, 0.5, n) * h0
    hv0 = rng.uniform(-0.5, 0.5, n) * h0
    return mi, h0, hu0, hv0


def test_mirror_symmetry_brute_force():
    # reflecting the mesh x -> -x and the x-momentum gives the reflected
    # solution (the oracle re-orients the mirrored triangles itself)
    mi, h0, hu0, hv0 = _mirror_case()
    A = _mesh(mi)
    nodes_m = mi.nodes * np.array([-1.0, 1.0])
    B = oracle.Mesh(nodes_m, mi.tris, mi.z, mi.manning)
    for pairs, kind, value in mi.bcs:
        B.set_bc(pairs, kind, value)
    ha, hua, hva, ta, _ = A.run(h0, hu0, hv0, 60, 0.9)
    hb, hub, hvb, tb, _ = B.run(h0, -hu0, hv0, 60, 0.9)
    assert tb == pytest.approx(ta, rel=1e-13)
    assert oracle.rel_err(hb, ha) < 1e-12
    assert oracle.rel_err(-hub, hua) < 1e-11
    assert oracle.rel_err(hvb, hva) < 1e-11


def test_rotation_invariance():
    # rotating mesh and velocities by theta rotates the solution (Eq 12)
    mi, h0, hu0, hv0 = _mirror_case()
    th = 0.7
    c, s = math.cos(th), math.sin(th)
    Rm = np.array([[c, -s], [s, c]])
    A = _mesh(mi)
    B = oracle.Mesh(mi.nodes @ Rm.T, mi.tris, mi.z, mi.manning)
    for pairs, kind, value in mi.bcs:
        B.set_bc(pairs, kind, value)
    ha, hua, hva, ta, _ = A.run(h0, hu0, hv0, 60, 0.9)
    hb, hub, hvb, tb, _ = B.run(h0, c * hu0 - s * hv0, s * hu0 + c * hv0, 60, 0.9)
    assert oracle.rel_err(hb, ha) < 1e-10
    assert oracle.rel_err(c * hua - s * hva, hub) < 1e-9
    assert oracle.rel_err(s * hua + c * hva, hvb) < 1e-9


def test_boundary_discharge_closed_forms_and_discrete_volume_balance():
    # inflow group carries exactly -Q outward, walls carry nothing, and the
    # stored volume changes by exactly -dt * (sum of outward discharges) in
    # one step, because interior fluxes cancel (Eq 9)
    mi = mg.river(60, 12, Lx=1200.0, Ly=240.0, seed=3, Q=150.0, n_bumps=10)
    M = _mesh(mi)
    area = M.geometry()["area"]
    h, hu, hv = mi.h, mi.hu, mi.hv
    for _ in range(30):
        Q = M.discharge(h, hu, hv)
        assert Q[0] == 0.0                                  # walls
        assert Q[1] == pytest.approx(-150.0, rel=1e-13)     # inflow
        dt = M.dt(h, hu, hv, 0.9)
        h2, hu2, hv2, c = M.step(h, hu, hv, dt)
        assert c == 0
        dV = (area * h2).sum() - (area * h).sum()
        assert dV == pytest.approx(-dt * Q.sum(), rel=1e-9, abs=1e-9 * (area * h).sum())
        h, hu, hv = h2, hu2, hv2
    # the outflow through the stage edge is positive once water reaches it
    mi2 = mg.canal(40, 4, 40.0, 4.0, 0.2, 2, hL=2.0, hR=2.0)
    M2 = oracle.Mesh(mi2.nodes, mi2.tris, mi2.z, mi2.manning)
    M2.set_bc(mg._side_pairs(40, 4)["right"].astype(np.int32), oracle.BC_STAGE, 1.0)
    assert M2.discharge(mi2.h, mi2.hu, mi2.hv)[1] > 0.0


def test_hll_scheme_conserves_and_balances():
    # the HLL variant keeps the well-balanced and conservative properties
    mi = mg.river(60, 12, seed=2, fully_wet=True)
    eta0 = mi.meta["eta0"]
    M = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    M.set_flux(1)
    M.set_bc(mi.bcs[1][0], oracle.BC_STAGE, eta0)
    h0 = np.maximum(eta0 - mi.z, 0.0)
    h, hu, hv, t, c = M.run(h0, np.zeros_like(h0), np.zeros_like(h0), 300, 0.9)
    assert np.abs(h + mi.z - eta0).max() < 1e-12 and np.abs(hu).max() < 1e-10
    mi = mg.dam_break_4k()
    M = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    M.set_flux(1)
    area = M.geometry()["area"]
    h, hu, hv, t, c = M.run(mi.h, mi.hu, mi.hv, 300, 0.9)
    assert abs((area * h).sum() - (area * mi.h).sum()) / (area * mi.h).sum() < 1e-13
    # HLL and HLLC differ only through the tangential momentum flux
    M2 = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    h2, hu2, hv2, t2, c2 = M2.run(mi.h, mi.hu, mi.hv, 300, 0.9)
    assert not np.array_equal(hv, hv2)


def test_quiet_cells_keep_their_depth_and_come_to_rest_exactly():
    # A dry cell (h <= h_dry) whose neighbours are all dry and whose boundary
    # edges are walls sees only mass fluxes of exactly zero (both Riemann
    # states dry, walls carry no mass): its depth is unchanged bit for bit and
    # the dry-cell rule leaves it at rest.  The GPU kernels' quiet path and
    # activity bytes skip such cells' fluxes on exactly this property.
    mi = mg.river(120, 24, seed=3)
    M = _mesh(mi)
    rng = np.random.default_rng(5)
    h = mi.h.copy()
    dry = h <= 1e-6
    h[dry] = rng.choice([0.0, 3e-7, 9e-7], size=int(dry.sum()))     # dry, some not exactly empty
    hu = mi.hu.copy()
    hv = mi.hv.copy()
    hu[dry] = rng.uniform(-1e-6, 1e-6, int(dry.sum()))             # stray momentum on dry cells
    hv[dry] = rng.uniform(-1e-6, 1e-6, int(dry.sum()))
    nbr = M.geometry()["nbr"]
    interior = nbr >= 0
    nbr_dry = np.where(interior, dry[np.where(interior, nbr, 0)], True).all(axis=1)
    walls_only = ((nbr >= 0) | (nbr == -1)).all(axis=1)               # -1: the wall group
    quiet = dry & nbr_dry & walls_only
    assert quiet.sum() > 1000 and (dry & ~quiet).sum() > 10          # both kinds of dry cell occur
    dt = M.dt(h, hu, hv, 0.9)
    h1, hu1, hv1, c = M.step(h, hu, hv, dt)
    assert c == 0
    assert np.array_equal(h1[quiet], h[quiet])
    assert np.all(hu1[quiet] == 0.0) and np.all(hv1[quiet] == 0.0)
