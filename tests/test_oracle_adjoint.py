"""Pins for the reference gradient (oracle/adjoint_torch.py): its forward map
equals the C oracle's, and its gradient of the gauge misfit matches central
differences of the C oracle with the time steps frozen, and forward-mode
directional derivatives (an independent differentiation of the same map)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import adjoint_torch as at  # noqa: E402
from paper_2010_14416_gb300 import meshgen as mg  # noqa: E402


def _case(fully_wet=True, seed=2, nx=40, ny=8, steps=80):
    mi = mg.river(nx, ny, Lx=2000.0, Ly=400.0, seed=seed, fully_wet=fully_wet, n_bumps=30, Q=300.0)
    M = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    for pairs, kind, value in mi.bcs:
        M.set_bc(pairs, kind, value)
    h, hu, hv, t, c, dts = M.run(mi.h, mi.hu, mi.hv, steps, 0.9, log_dt=True)
    gauges = mg.gauge_cells(mi.n_cells, 12, seed=seed)
    xi = mg.perturbation(mi.n_cells, seed + 100)
    # target: the same run with perturbed Manning and bed (its own CFL steps)
    T = oracle.Mesh(mi.nodes, mi.tris, mi.z + 0.05 * xi, mi.manning * (1 + 0.1 * xi))
    for pairs, kind, value in mi.bcs:
        T.set_bc(pairs, kind, value)
    th, _, _, _, _ = T.run(mi.h, mi.hu, mi.hv, steps, 0.9)
    return mi, M, dts, gauges, th[gauges], h


@pytest.mark.parametrize("fully_wet", [True, False])
def test_torch_forward_equals_c_oracle(fully_wet):
    mi, M, dts, gauges, target, h_c = _case(fully_wet)
    step = at.TorchStep(M)
    with torch.no_grad():
        h, hu, hv = at.run(step, *(torch.tensor(a) for a in (mi.h, mi.hu, mi.hv)),
                           torch.tensor(M.z), torch.tensor(M.m), dts)
    hc, huc, hvc, _ = M.run_fixed_dt(mi.h, mi.hu, mi.hv, dts)
    assert oracle.rel_err(h.numpy(), hc) < 1e-12
    assert oracle.rel_err(hu.numpy(), huc) < 1e-11
    assert oracle.rel_err(hv.numpy(), hvc) < 1e-11


def test_gradient_matches_central_differences_of_c_oracle():
    mi, M, dts, gauges, target, _ = _case(True)
    L0, gm, gz = at.loss_and_gradient(M, mi.h, mi.hu, mi.hv, dts, gauges, target)
    assert L0 > 0
    rng = np.random.default_rng(9)

    def c_loss(z, m):
        M.set_fields(z=z, m=m)
        h, _, _, _ = M.run_fixed_dt(mi.h, mi.hu, mi.hv, dts)
        return float(((h[gauges] - target) ** 2).sum())

    z0, m0 = mi.z.copy(), mi.manning.copy()
    for _ in range(4):
        vz = rng.standard_normal(mi.n_cells)
        vm = 0.01 * rng.standard_normal(mi.n_cells)
        eps = 1e-4
        fd = (c_loss(z0 + eps * vz, m0 + eps * vm) - c_loss(z0 - eps * vz, m0 - eps * vm)) / (2 * eps)
        ad = float(gz @ vz + gm @ vm)
        assert abs(fd - ad) <= 1e-6 * max(abs(ad), 1e-12) + 1e-13, (fd, ad)
    M.set_fields(z=z0, m=m0)


def test_reverse_gradient_matches_forward_mode():
    mi, M, dts, gauges, target, _ = _case(True, steps=40)
    L0, gm, gz = at.loss_and_gradient(M, mi.h, mi.hu, mi.hv, dts, gauges, target)
    step = at.TorchStep(M)
    h0, hu0, hv0 = (torch.tensor(a) for a in (mi.h, mi.hu, mi.hv))
    gi = torch.tensor(gauges.astype(np.int64))
    tt = torch.tensor(target)

    def loss(z, m):
        h, hu, hv = h0, hu0, hv0
        for dt in dts:
            h, hu, hv = step.step(h, hu, hv, z, m, float(dt))
        return ((h[gi] - tt) ** 2).sum()

    rng = np.random.default_rng(4)
    for _ in range(3):
        vz = torch.tensor(rng.standard_normal(mi.n_cells))
        vm = torch.tensor(0.01 * rng.standard_normal(mi.n_cells))
        _, d = torch.func.jvp(loss, (torch.tensor(M.z), torch.tensor(M.m)), (vz, vm))
        ad = float(gz @ vz.numpy() + gm @ vm.numpy())
        assert abs(float(d) - ad) <= 1e-10 * max(abs(ad), 1e-12), (float(d), ad)


def _series_targets(mi, steps, every, seed=2):
    xi = mg.perturbation(mi.n_cells, seed + 100)
    T = oracle.Mesh(mi.nodes, mi.tris, mi.z + 0.05 * xi, mi.manning * (1 + 0.1 * xi))
    for pairs, kind, value in mi.bcs:
        T.set_bc(pairs, kind, value)
    h, hu, hv = mi.h, mi.hu, mi.hv
    out = []
    for _ in range(steps // every):
        h, hu, hv, _, _ = T.run(h, hu, hv, every, 0.9)
        out.append(h)
    return np.array(out)


def test_series_reference_reduces_to_final_loss_and_matches_differences():
    mi, M, dts, gauges, target, _ = _case(True, steps=60)
    L1, gm1, gz1 = at.loss_and_gradient(M, mi.h, mi.hu, mi.hv, dts, gauges, target)
    L2, gm2, gz2 = at.loss_and_gradient_series(M, mi.h, mi.hu, mi.hv, dts, gauges, target[None, :], 60)
    assert L2 == pytest.approx(L1, rel=1e-14)
    assert np.allclose(gm2, gm1, rtol=1e-12, atol=0) and np.allclose(gz2, gz1, rtol=1e-12, atol=0)
    targets = _series_targets(mi, 60, 20)[:, gauges]
    L, gm, gz = at.loss_and_gradient_series(M, mi.h, mi.hu, mi.hv, dts, gauges, targets, 20)

    def c_loss(z, m):
        M.set_fields(z=z, m=m)
        h, hu, hv = mi.h, mi.hu, mi.hv
        tot = 0.0
        for o in range(3):
            h, hu, hv, _ = M.run_fixed_dt(h, hu, hv, dts[20 * o:20 * (o + 1)])
            tot += float(((h[gauges] - targets[o]) ** 2).sum())
        return tot

    rng = np.random.default_rng(3)
    z0, m0 = mi.z.copy(), mi.manning.copy()
    assert c_loss(z0, m0) == pytest.approx(L, rel=1e-10)
    for _ in range(3):
        vz = rng.standard_normal(mi.n_cells)
        vm = 0.01 * rng.standard_normal(mi.n_cells)
        eps = 1e-4
        fd = (c_loss(z0 + eps * vz, m0 + eps * vm) - c_loss(z0 - eps * vz, m0 - eps * vm)) / (2 * eps)
        ad = float(gz @ vz + gm @ vm)
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    M.set_fields(z=z0, m=m0)
