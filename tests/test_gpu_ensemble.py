"""Batched ensemble (uncertainty propagation, Section 6.4.3's sampled runs):
members of uneven sizes advanced together must receive exactly the updates
the plain solver gives each of them alone, bit for bit, with their own CFL
steps."""
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


def _members(n=8, seed=3):
    return mg.ensemble_members(n, seed=seed, lo=1500, hi=30000)


def _mesh(mi, precision, **kw):
    m = capi.Mesh(mi.nodes, mi.tris, mi.z, mi.manning, precision=precision, **kw)
    for pairs, kind, value in mi.bcs:
        m.set_bc(pairs, kind, value)
    dt = m.dtype
    m.set_state(mi.h.astype(dt), mi.hu.astype(dt), mi.hv.astype(dt))
    return m


@pytest.mark.parametrize("precision", [capi.SWE_FP64, capi.SWE_FP32])
def test_ensemble_matches_plain_solver_bitwise(precision):
    mis = _members()
    assert len({mi.n_cells % 256 for mi in mis}) > 1          # uneven, ragged sizes
    rng = np.random.default_rng(1)
    cfl = rng.uniform(0.5, 0.9, len(mis))
    meshes = [_mesh(mi, precision) for mi in mis]
    ens = capi.Ensemble(meshes)
    t_a = ens.step(100, cfl)
    t_b = ens.step(101, cfl)                                   # second call starts mid-phase
    for k, (mi, m) in enumerate(zip(mis, meshes)):
        t_plain = m.step(201, cfl[k])
        assert t_b[k] == t_plain and t_a[k] < t_b[k]
        got = ens.get_state(k)
        ref = m.get_state()
        assert all(np.array_equal(a, b) for a, b in zip(got, ref)), f"member {k}"
        assert ens.info(k)["status"] == 0
    ens.close()
    for m in meshes:
        m.close()


def test_ensemble_member_against_oracle_fp64():
    mis = _members(4, seed=5)
    meshes = [_mesh(mi, capi.SWE_FP64) for mi in mis]
    ens = capi.Ensemble(meshes)
    t = ens.step(300)
    for k in (0, 3):
        mi = mis[k]
        M = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
        for pairs, kind, value in mi.bcs:
            M.set_bc(pairs, kind, value)
        oh, ohu, ohv, ot, _ = M.run(mi.h, mi.hu, mi.hv, 300, 0.9)
        assert t[k] == pytest.approx(ot, rel=1e-12)
        for a, b in zip(ens.get_state(k), (oh, ohu, ohv)):
            assert rel_err(a, b) <= 1e-10
    ens.close()


def test_ensemble_device_output_and_errors():
    mis = _members(3, seed=7)
    meshes = [_mesh(mi, capi.SWE_FP64) for mi in mis]
    ens = capi.Ensemble(meshes)
    ens.step(12)
    out = [torch.empty(mis[1].n_cells, dtype=torch.float64, device="cuda") for _ in range(3)]
    ens.get_state(1, out)
    torch.cuda.synchronize()
    host = ens.get_state(1)
    assert all(np.array_equal(a.cpu().numpy(), b) for a, b in zip(out, host))
    ens.close()
    # a member without a state, or of another precision, is refused
    bare = capi.Mesh(mis[0].nodes, mis[0].tris, mis[0].z, mis[0].manning)
    with pytest.raises(capi.SWEError) as e:
        capi.Ensemble([meshes[0], bare])
    assert e.value.code == capi.SWE_EINVAL
    f32 = _mesh(mis[0], capi.SWE_FP32)
    with pytest.raises(capi.SWEError) as e:
        capi.Ensemble([meshes[0], f32])
    assert e.value.code == capi.SWE_EINVAL


@pytest.mark.parametrize("precision", [capi.SWE_FP64, capi.SWE_FP32])
def test_ensemble_launch_shapes_are_bitwise_neutral(precision):
    # every batched kernel shape -- tile size, staging, geometry placement,
    # activity bytes, chunk, grid and (FP32) the split step over cell pairs and
    # the per-warp queues -- gives each member the plain solver's updates bit
    # for bit, also when the shape changes between calls
    mis = _members(6, seed=13)
    meshes = [_mesh(mi, precision) for mi in mis]
    ens = capi.Ensemble(meshes)
    f32 = precision == capi.SWE_FP32
    shapes = [dict(block_size=128, min_blocks=8 if f32 else 1, activity=1, chunk=4),
              dict(block_size=256, min_blocks=4 if f32 else 1, activity=1, chunk=16, grid=37),
              dict(block_size=256, min_blocks=4 if f32 else 1, stages=3 if f32 else 1, chunk=8),
              dict(block_size=128, min_blocks=8 if f32 else 1, geometry_early=1 if f32 else 0, activity=1,
                   chunk=64, grid=5)]
    # chunks taken dynamically from a per-step counter, switched to and from
    shapes += [dict(block_size=128, min_blocks=8 if f32 else 1, dynamic=1, chunk=1),
               dict(block_size=256, min_blocks=4 if f32 else 1, stages=3 if f32 else 1, chunk=4),
               dict(block_size=256, min_blocks=4 if f32 else 1, dynamic=1, chunk=8, grid=17)]
    # activity bytes with dynamically taken chunks (at least 4 tiles)
    shapes += [dict(block_size=128, min_blocks=8 if f32 else 1, activity=1, dynamic=1, chunk=4),
               dict(block_size=256, min_blocks=4 if f32 else 1, activity=1, dynamic=1, chunk=32, grid=23),
               dict(block_size=128, min_blocks=8 if f32 else 1, geometry_early=1 if f32 else 0, activity=1,
                    dynamic=1, chunk=8, grid=3)]
    if not f32:   # the edge pass of FP64 ensembles
        shapes += [dict(block_size=256, min_blocks=1, edge_pass=1, chunk=8),
                   dict(block_size=128, min_blocks=1, edge_pass=1, chunk=4, grid=11)]
    else:   # split steps: the members wet at creation on the cell-pair kernel, the rest on the given one
        shapes += [dict(block_size=128, min_blocks=8, activity=1, dynamic=1, chunk=4, cell_pairs=1),
                   dict(block_size=256, min_blocks=4, activity=1, chunk=16, grid=37, cell_pairs=1),
                   dict(block_size=128, min_blocks=8, dynamic=1, chunk=1, cell_pairs=1),
                   dict(block_size=256, min_blocks=4, stages=3, chunk=8, cell_pairs=1),
                   dict(block_size=128, min_blocks=8, geometry_early=1, activity=1, chunk=64, grid=5, cell_pairs=1)]
        # per-warp queues of the cells that run the flux path, alone and in split steps
        shapes += [dict(block_size=128, min_blocks=7, geometry_early=1, activity=1, chunk=8, queue=1),
                   dict(block_size=128, min_blocks=7, activity=1, dynamic=1, chunk=4, grid=9, queue=1, cell_pairs=1),
                   dict(block_size=128, min_blocks=6, geometry_early=1, activity=1, dynamic=1, chunk=16, queue=1),
                   dict(block_size=128, min_blocks=7, geometry_early=1, activity=1, chunk=4, grid=3, queue=1,
                        cell_pairs=1)]
    steps = 0
    for k, sh in enumerate(shapes):
        ens.set_shape(**sh)
        ens.step(37 + k)
        steps += 37 + k
    t_ens = ens.step(0)
    for k, m in enumerate(meshes):
        assert m.step(steps) == t_ens[k]
        assert all(np.array_equal(a, b) for a, b in zip(ens.get_state(k), m.get_state())), f"member {k}"
    assert ens.info(0)["n_active"] == sum(m.info()["n_active"] for m in meshes)
    with pytest.raises(capi.SWEError):
        ens.set_shape(block_size=512, min_blocks=2, activity=1)
    with pytest.raises(capi.SWEError):
        ens.set_shape(block_size=256, min_blocks=4 if f32 else 1, activity=1, edge_pass=1)
    with pytest.raises(capi.SWEError):   # dynamic activity chunks hold at least 4 tiles
        ens.set_shape(block_size=128, min_blocks=8 if f32 else 1, activity=1, dynamic=1, chunk=2)
    with pytest.raises(capi.SWEError):
        ens.set_shape(block_size=256, min_blocks=4 if f32 else 1, dynamic=1, edge_pass=1)
    if not f32:   # the split step and the queues are FP32 only
        with pytest.raises(capi.SWEError):
            ens.set_shape(block_size=128, min_blocks=1, activity=1, chunk=4, cell_pairs=1)
        with pytest.raises(capi.SWEError):
            ens.set_shape(block_size=128, min_blocks=1, activity=1, chunk=4, queue=1)
    else:   # queues need the activity kernel
        with pytest.raises(capi.SWEError):
            ens.set_shape(block_size=128, min_blocks=7, dynamic=1, chunk=4, queue=1)
    ens.close()
    for m in meshes:
        m.close()


@pytest.mark.parametrize("precision", [capi.SWE_FP64, capi.SWE_FP32])
def test_ensemble_debug_checks_change_nothing(precision):
    # members created with debug checks: the batched kernels check every
    # index and boundary group before use; a valid ensemble steps exactly as
    # without them, with status 0
    mis = _members(4, seed=9)
    ref_meshes = [_mesh(mi, precision) for mi in mis]
    ref = capi.Ensemble(ref_meshes)
    t_ref = ref.step(120)
    dbg_meshes = [_mesh(mi, precision, debug_checks=1) for mi in mis]
    dbg = capi.Ensemble(dbg_meshes)
    shapes = [None, dict(block_size=128, min_blocks=8 if precision == capi.SWE_FP32 else 1, activity=1, chunk=4)]
    if precision == capi.SWE_FP64:
        shapes.append(dict(block_size=256, min_blocks=1, edge_pass=1, chunk=4))
    else:
        shapes.append(dict(block_size=128, min_blocks=8, activity=1, dynamic=1, chunk=4, cell_pairs=1))
        shapes.append(dict(block_size=128, min_blocks=7, geometry_early=1, activity=1, chunk=4, queue=1))
    for shape in shapes:
        for k, m in enumerate(dbg_meshes):
            m.set_state(*(a.astype(m.dtype) for a in (mis[k].h, mis[k].hu, mis[k].hv)))
        dbg.close()
        dbg = capi.Ensemble(dbg_meshes)
        if shape:
            dbg.set_shape(**shape)
        t = dbg.step(120)
        assert np.array_equal(t, t_ref), shape
        for k in range(len(mis)):
            assert dbg.info(k)["status"] == 0
            assert all(np.array_equal(a, b) for a, b in zip(dbg.get_state(k), ref.get_state(k))), (shape, k)
    for e in (ref, dbg):
        e.close()
    for m in ref_meshes + dbg_meshes:
        m.close()
