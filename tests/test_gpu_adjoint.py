"""Discrete adjoint (gradient of the gauge misfit w.r.t. Manning n and bed
elevation) against the FP64 reference gradient of oracle/adjoint_torch.py,
against central differences of the GPU's own frozen-dt forward map, and
through the torch.autograd.Function."""
import numpy as np
import pytest

import oracle
from oracle import adjoint_torch as at
from paper_2010_14416_gb300 import build as libbuild
from paper_2010_14416_gb300 import capi
from paper_2010_14416_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    libbuild.build()
    return capi.load()


def _setup(fully_wet=True, nx=40, ny=8, steps=80, seed=2, n_gauges=12):
    mi = mg.river(nx, ny, Lx=50.0 * nx, Ly=50.0 * ny, seed=seed, fully_wet=fully_wet, n_bumps=30, Q=300.0)
    M = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    for pairs, kind, value in mi.bcs:
        M.set_bc(pairs, kind, value)
    _, _, _, _, _, dts = M.run(mi.h, mi.hu, mi.hv, steps, 0.9, log_dt=True)
    if fully_wet:
        gauges = mg.gauge_cells(mi.n_cells, n_gauges, seed=seed)
    else:  # gauges in the wet channel, so the misfit depends on the parameters
        wet = np.flatnonzero(mi.h > 0.5)
        gauges = np.sort(wet[mg.gauge_cells(wet.shape[0], n_gauges, seed=seed)])
    xi = mg.perturbation(mi.n_cells, seed + 100)
    T = oracle.Mesh(mi.nodes, mi.tris, mi.z + 0.05 * xi, mi.manning * (1 + 0.1 * xi))
    for pairs, kind, value in mi.bcs:
        T.set_bc(pairs, kind, value)
    th, _, _, _, _ = T.run(mi.h, mi.hu, mi.hv, steps, 0.9)
    return mi, M, dts, gauges, th[gauges]


def _gpu_mesh(mi, **kw):
    m = capi.Mesh(mi.nodes, mi.tris, mi.z, mi.manning, precision=capi.SWE_FP64, **kw)
    for pairs, kind, value in mi.bcs:
        m.set_bc(pairs, kind, value)
    m.set_state(mi.h, mi.hu, mi.hv)
    return m


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("fully_wet,ckpt", [(True, 50), (True, 7), (False, 50)])
def test_adjoint_matches_reference_gradient(fully_wet, ckpt):
    mi, M, dts, gauges, target = _setup(fully_wet)
    L_ref, gm_ref, gz_ref = at.loss_and_gradient(M, mi.h, mi.hu, mi.hv, dts, gauges, target)
    m = _gpu_mesh(mi)
    L, gm, gz, gdts = m.adjoint(len(dts), gauges, target, cfl=0.9, checkpoint_every=ckpt)
    assert np.allclose(gdts, dts, rtol=1e-12)
    assert L == pytest.approx(L_ref, rel=1e-9)
    assert _rel(gm, gm_ref) <= TOL
    assert _rel(gz, gz_ref) <= TOL
    # the mesh state advanced to U^N like swe_step
    assert m.info()["n_steps"] == len(dts)
    m.close()


def test_adjoint_directional_derivatives_match_central_differences():
    # The discrete map has tiny jumps where the h* estimate switches between
    # its rarefaction and shock forms (Eq 22/23), so differences use a small
    # step that rarely straddles a switch; the full gradient is also checked
    # against the reference gradient on the same case.
    mi, M, dts, gauges, target = _setup(True, nx=120, ny=24, steps=150, seed=4, n_gauges=32)
    m = _gpu_mesh(mi)
    L0, gm, gz, gdts = m.adjoint(len(dts), gauges, target, checkpoint_every=50)
    L_ref, gm_ref, gz_ref = at.loss_and_gradient(M, mi.h, mi.hu, mi.hv, dts, gauges, target)
    assert _rel(gm, gm_ref) <= TOL and _rel(gz, gz_ref) <= TOL
    rng = np.random.default_rng(12)

    def loss(z, man):
        m.set_fields(bathy=z, manning=man)
        m.set_state(mi.h, mi.hu, mi.hv)
        m.step_dt(gdts)
        h, _, _ = m.get_state()
        return float(((h[gauges] - target) ** 2).sum())

    errs = []
    for _ in range(32):
        vz = rng.standard_normal(mi.n_cells)
        vm = 0.01 * rng.standard_normal(mi.n_cells)
        eps = 1e-6
        fd = (loss(mi.z + eps * vz, mi.manning + eps * vm) - loss(mi.z - eps * vz, mi.manning - eps * vm)) / (2 * eps)
        ad = float(gz @ vz + gm @ vm)
        errs.append(abs(fd - ad) / abs(ad))
    errs = np.array(errs)
    assert np.median(errs) <= TOL, errs
    assert (errs <= 1e-5).mean() >= 0.9, errs
    m.close()


def test_autograd_function():
    from paper_2010_14416_gb300.autograd import SWEAdjoint
    mi, M, dts, gauges, target = _setup(True, steps=40)
    m = _gpu_mesh(mi)
    man = torch.tensor(mi.manning, device="cuda", requires_grad=True)
    bed = torch.tensor(mi.z, device="cuda", requires_grad=True)
    loss = SWEAdjoint.apply(man, bed, m, (mi.h, mi.hu, mi.hv), 40, gauges, target)
    (3.0 * loss).backward()
    L_ref, gm_ref, gz_ref = at.loss_and_gradient(M, mi.h, mi.hu, mi.hv, dts[:40], gauges, target)
    assert float(loss.detach()) == pytest.approx(L_ref, rel=1e-9)
    assert _rel(man.grad.cpu().numpy(), 3.0 * gm_ref) <= TOL
    assert _rel(bed.grad.cpu().numpy(), 3.0 * gz_ref) <= TOL
    m.close()


@pytest.mark.parametrize("fully_wet,flux", [(True, capi.SWE_FLUX_HLLC), (False, capi.SWE_FLUX_HLLC),
                                             (True, capi.SWE_FLUX_HLL)])
def test_adjoint_transposes_match_dual_number_kernels(fully_wet, flux):
    # the hand-written transposes of the edge terms (the default reverse step,
    # each interior edge once) against the dual-number reverse step (each edge
    # from both cells on forward-mode duals): the same discrete derivative,
    # through wet/dry fronts and both fluxes
    mi, M, dts, gauges, target = _setup(fully_wet, nx=60, ny=12, steps=60)
    res = {}
    for method in (capi.SWE_ADJOINT_TRANSPOSE, capi.SWE_ADJOINT_DUAL):
        m = _gpu_mesh(mi, flux=flux)
        m.adjoint_method(method)
        res[method] = m.adjoint(60, gauges, target, checkpoint_every=7)
        m.close()
    a, b = res[capi.SWE_ADJOINT_TRANSPOSE], res[capi.SWE_ADJOINT_DUAL]
    assert a[0] == b[0]                      # the same forward run and loss
    assert np.array_equal(a[3], b[3])
    assert _rel(a[1], b[1]) <= 1e-12 and _rel(a[2], b[2]) <= 1e-12, (_rel(a[1], b[1]), _rel(a[2], b[2]))


def test_adjoint_method_is_checked():
    mi = mg.river(20, 4, seed=1, fully_wet=True)
    m = _gpu_mesh(mi)
    with pytest.raises(capi.SWEError) as e:
        m.adjoint_method(2)
    assert e.value.code == capi.SWE_EINVAL
    m.close()


def test_adjoint_with_debug_checks_is_unchanged():
    # the adjoint kernels check their neighbour codes and edge indices too; on
    # a valid mesh nothing changes, with the edge pass and without
    mi, M, dts, gauges, target = _setup(True, steps=40)
    for kw in (dict(), dict(edge_pass=1)):
        ref = _gpu_mesh(mi, **kw).adjoint(40, gauges, target, checkpoint_every=7)
        got = _gpu_mesh(mi, debug_checks=1, **kw).adjoint(40, gauges, target, checkpoint_every=7)
        assert got[0] == ref[0], kw
        assert all(np.array_equal(a, b) for a, b in zip(got[1:], ref[1:])), kw


def test_adjoint_refuses_fp32_and_bad_gauges():
    mi = mg.river(20, 4, seed=1, fully_wet=True)
    m32 = capi.Mesh(mi.nodes, mi.tris, mi.z, mi.manning, precision=capi.SWE_FP32)
    m32.set_state(mi.h.astype(np.float32), mi.hu.astype(np.float32), mi.hv.astype(np.float32))
    with pytest.raises(capi.SWEError) as e:
        m32.adjoint(5, [0], [1.0])
    assert e.value.code == capi.SWE_EINVAL
    m = _gpu_mesh(mi)
    with pytest.raises(capi.SWEError) as e:
        m.adjoint(5, [mi.n_cells], [1.0])
    assert e.value.code == capi.SWE_EINVAL


def _c24_target(mi, gauges, steps, seed=101):
    """The workload's seeded target (the oracle's run of the same mesh with
    Manning m (1 + 0.1 xi) and bed z + 0.05 xi, xi ~ N(0, 1)) at the gauges."""
    xi = mg.perturbation(mi.n_cells, seed)
    T = oracle.Mesh(mi.nodes, mi.tris, mi.z + 0.05 * xi, mi.manning * (1 + 0.1 * xi))
    for pairs, kind, value in mi.bcs:
        T.set_bc(pairs, kind, value)
    th, _, _, _, _ = T.run(mi.h, mi.hu, mi.hv, steps, 0.9)
    return th[gauges]


def test_adjoint_at_the_workload_length_matches_reference_gradient():
    # the adjoint workload's length and settings on a 20,224-cell copy of its
    # reach: 2000 FP64 steps, 64 seeded gauges, checkpoints every 50 steps, the
    # seeded perturbed-parameter target; the gradients with respect to Manning
    # n and to the bed, each against the reference gradient of the plain
    # PyTorch FP64 statement of the scheme
    mi = mg.river_adjoint_20k()
    M = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    for pairs, kind, value in mi.bcs:
        M.set_bc(pairs, kind, value)
    _, _, _, _, _, dts = M.run(mi.h, mi.hu, mi.hv, 2000, 0.9, log_dt=True)
    gauges = mg.gauge_cells(mi.n_cells, 64, seed=1)
    target = _c24_target(mi, gauges, 2000)
    L_ref, gm_ref, gz_ref = at.loss_and_gradient(M, mi.h, mi.hu, mi.hv, dts, gauges, target)
    # water flows past the gauges, so the Manning gradient is far above round-off
    assert np.linalg.norm(gm_ref) > 1e-2 * np.linalg.norm(gz_ref)
    m = _gpu_mesh(mi)
    L, gm, gz, gdts = m.adjoint(2000, gauges, target, cfl=0.9, checkpoint_every=50)
    m.close()
    assert np.allclose(gdts, dts, rtol=1e-12)
    assert L == pytest.approx(L_ref, rel=1e-9)
    err_m, err_z = _rel(gm, gm_ref), _rel(gz, gz_ref)
    print(f"20k reach, 2000 steps: |dL/dn| {np.linalg.norm(gm_ref):.3e} rel err {err_m:.2e}; "
          f"|dL/dz| {np.linalg.norm(gz_ref):.3e} rel err {err_z:.2e}")
    assert err_m <= TOL and err_z <= TOL


def test_full_size_adjoint_1m_cells_2000_steps():
    # the adjoint workload itself: 1,001,728 cells, 2000 FP64 steps, 64
    # gauges, checkpoints every 50, the oracle's seeded perturbed-parameter
    # target; directional derivatives against central differences of the
    # frozen-dt map (a property that holds at any size), on 16 directions in
    # the bed alone and 16 in the Manning coefficients alone
    mi = mg.river_adjoint_1m()
    gauges = mg.gauge_cells(mi.n_cells, 64, seed=1)
    target = _c24_target(mi, gauges, 2000)
    m = _gpu_mesh(mi)
    L0, gm, gz, dts = m.adjoint(2000, gauges, target, checkpoint_every=50)
    assert np.isfinite(L0) and L0 > 0 and np.all(np.isfinite(gm)) and np.all(np.isfinite(gz))
    h_end, _, _ = m.get_state()
    assert float(((h_end[gauges] - target) ** 2).sum()) == pytest.approx(L0, rel=1e-12)
    assert np.linalg.norm(gm) > 1e-3 * np.linalg.norm(gz)
    rng = np.random.default_rng(3)

    def loss(z, man):
        m.set_fields(bathy=z, manning=man)
        m.set_state(mi.h, mi.hu, mi.hv)
        m.step_dt(dts)
        h, _, _ = m.get_state()
        return float(((h[gauges] - target) ** 2).sum())

    errs = {"bed": [], "manning": []}
    for k in range(32):   # 32 random directions, as the workload asks
        part = "bed" if k % 2 == 0 else "manning"
        v = rng.standard_normal(mi.n_cells)
        if part == "bed":
            eps = 1e-6
            fd = (loss(mi.z + eps * v, mi.manning) - loss(mi.z - eps * v, mi.manning)) / (2 * eps)
            ad = float(gz @ v)
        else:
            v *= 0.01
            eps = 1e-4
            fd = (loss(mi.z, mi.manning + eps * v) - loss(mi.z, mi.manning - eps * v)) / (2 * eps)
            ad = float(gm @ v)
        errs[part].append(abs(fd - ad) / abs(ad))
    m.close()
    print("full-size directional derivative errors:",
          {k: (float(np.median(v)), float(np.max(v))) for k, v in errs.items()})
    for part, e in errs.items():
        e = np.array(e)
        assert np.median(e) <= 1e-5, (part, e)
        assert (e <= 1e-4).mean() >= 0.9, (part, e)


def test_adjoint_time_series_matches_reference_gradient():
    from tests.test_oracle_adjoint import _series_targets
    mi, M, dts, gauges, target = _setup(True, steps=90)
    targets = _series_targets(mi, 90, 30)[:, gauges]
    L_ref, gm_ref, gz_ref = at.loss_and_gradient_series(M, mi.h, mi.hu, mi.hv, dts, gauges, targets, 30)
    m = _gpu_mesh(mi)
    L, gm, gz, _ = m.adjoint_series(90, gauges, targets, 30, checkpoint_every=20)
    assert L == pytest.approx(L_ref, rel=1e-9)
    assert _rel(gm, gm_ref) <= TOL and _rel(gz, gz_ref) <= TOL
    m.close()


@pytest.mark.parametrize("fully_wet", [True, False])
def test_adjoint_is_independent_of_the_forward_launch_shape(fully_wet):
    # the forward and recomputed steps of the adjoint run the mesh's shape for
    # launches outside the step loop (the edge pass here, or whatever the
    # autotuner keeps): loss, gradients and step sizes are bit for bit those
    # of the default shape
    mi, M, dts, gauges, target = _setup(fully_wet, steps=60)
    ref = _gpu_mesh(mi).adjoint(60, gauges, target, checkpoint_every=7)
    got = _gpu_mesh(mi, edge_pass=1).adjoint(60, gauges, target, checkpoint_every=7)
    assert got[0] == ref[0]
    for a, b in zip(got[1:], ref[1:]):
        assert np.array_equal(a, b)
    tuned = _gpu_mesh(mi)
    tuned.autotune(trial_steps=2)
    got = tuned.adjoint(60, gauges, target, checkpoint_every=7)
    assert got[0] == ref[0] and all(np.array_equal(a, b) for a, b in zip(got[1:], ref[1:]))
