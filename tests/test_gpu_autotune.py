"""Launch-shape autotuner (swe_autotune, swe_ensemble_autotune): the timing
calls leave every state, time and step count as they were, and whatever
shape they choose, the steps that follow are bit for bit those of the
default shape."""
import numpy as np
import pytest

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


def _mesh(mi, precision, **kw):
    m = capi.Mesh(mi.nodes, mi.tris, mi.z, mi.manning, precision=precision, **kw)
    for pairs, kind, value in mi.bcs:
        m.set_bc(pairs, kind, value)
    dt = m.dtype
    m.set_state(mi.h.astype(dt), mi.hu.astype(dt), mi.hv.astype(dt))
    return m


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


# (block, min_blocks, stages, geometry_early, activity)
F32_SHAPES = {s + (0,) for s in [
    (128, 1, 1, 0), (256, 1, 1, 0), (512, 1, 1, 0), (128, 8, 1, 0), (256, 4, 1, 0), (256, 5, 1, 0), (512, 2, 1, 0),
    (256, 4, 2, 0), (256, 4, 3, 0), (256, 4, 4, 0), (128, 8, 3, 0), (128, 8, 4, 0), (256, 4, 1, 1), (256, 4, 3, 1),
    (128, 8, 1, 1), (128, 8, 3, 1)]} | {
    (128, 8, 3, 0, 1), (256, 4, 3, 0, 1), (512, 2, 3, 0, 1), (128, 8, 3, 1, 1), (256, 4, 3, 1, 1),
    (128, 8, 4, 1, 1), (128, 8, 5, 1, 1), (256, 4, 4, 1, 1), (128, 8, 4, 0, 1)}
F64_SHAPES = {s + (0,) for s in [
    (128, 1, 1, 0), (256, 1, 1, 0), (512, 1, 1, 0), (128, 1, 2, 0), (256, 1, 2, 0), (128, 1, 1, 1), (256, 1, 1, 1)]} | {
    (128, 1, 3, 0, 1), (256, 1, 3, 0, 1), (128, 1, 3, 1, 1), (128, 1, 4, 0, 1)}
# (block, min_blocks, stages, geometry_early) of the edge pass's cell kernel
EDGE_CELL_PASS = {capi.SWE_FP32: {(256, 4, 1, 0), (128, 8, 1, 0)}, capi.SWE_FP64: {(128, 1, 1, 0), (256, 1, 1, 0)}}


@pytest.mark.parametrize("precision,maker", [(capi.SWE_FP64, "dam"), (capi.SWE_FP32, "dam"),
                                             (capi.SWE_FP32, "river")])
def test_mesh_autotune_keeps_state_and_results(precision, maker):
    mi = mg.dam_break_4k() if maker == "dam" else mg.river(160, 24, seed=4, n_bumps=20)
    tuned, plain = _mesh(mi, precision), _mesh(mi, precision)
    tuned.step(37)
    plain.step(37)
    before, info0 = tuned.get_state(), tuned.info()
    ch = tuned.autotune(trial_steps=3)
    after, info1 = tuned.get_state(), tuned.info()
    assert _same(before, after)
    assert info1["t"] == info0["t"] and info1["n_steps"] == info0["n_steps"]
    assert info1["dt_next"] == info0["dt_next"] and info1["n_active"] == info0["n_active"]
    shapes = F32_SHAPES if precision == capi.SWE_FP32 else F64_SHAPES
    key = (ch["block_size"], ch["min_blocks"], ch["stages"], ch["geometry_early"], ch["activity"])
    assert key in shapes if ch["edge_pass"] == 0 else key[:4] in EDGE_CELL_PASS[precision]
    assert not (ch["edge_pass"] and ch["activity"])
    assert ch["n_candidates"] > len(shapes) and ch["chunk"] == 0
    assert 0 < ch["ms_best"] <= ch["ms_before"]
    assert ch["grid"] >= 1
    assert ch["cells_per_thread"] == pytest.approx(mi.n_cells / (ch["grid"] * ch["block_size"]))
    # stepping on, through graphs and single launches, matches the untuned mesh bit for bit
    assert tuned.step(101) == plain.step(101)
    assert _same(tuned.get_state(), plain.get_state())
    assert tuned.info()["n_active"] == plain.info()["n_active"]


def test_mesh_autotune_rejects_missing_state():
    mi = mg.dam_break_4k()
    m = capi.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    with pytest.raises(capi.SWEError):
        m.autotune()


@pytest.mark.parametrize("precision", [capi.SWE_FP64, capi.SWE_FP32])
def test_ensemble_autotune_keeps_state_and_results(precision):
    mis = mg.ensemble_members(6, seed=11, lo=1500, hi=30000)
    rng = np.random.default_rng(2)
    cfl = rng.uniform(0.5, 0.9, len(mis))
    meshes = [_mesh(mi, precision) for mi in mis]
    ens = capi.Ensemble(meshes)
    ens.step(13, cfl)
    before = [ens.get_state(k) for k in range(len(mis))]
    infos = [ens.info(k) for k in range(len(mis))]
    ch = ens.autotune(trial_steps=2)
    for k in range(len(mis)):
        assert _same(before[k], ens.get_state(k))
        inf = ens.info(k)
        assert inf["t"] == infos[k]["t"] and inf["dt_next"] == infos[k]["dt_next"]
        assert inf["n_active"] == infos[k]["n_active"]
    assert ch["block_size"] in (128, 256) and ch["chunk"] in (1, 2, 4, 8, 16, 32, 64)
    assert ch["geometry_early"] in (0, 1) and ch["activity"] in (0, 1) and ch["edge_pass"] in (0, 1)
    assert not (ch["activity"] and ch["edge_pass"])
    assert ch["edge_pass"] == 0 or precision == capi.SWE_FP64
    assert ch["dynamic"] in (0, 1) and not (ch["edge_pass"] and (ch["activity"] or ch["dynamic"]))
    assert not (ch["activity"] and ch["dynamic"]) or ch["chunk"] >= 4
    assert ch["cell_pairs"] in (0, 1) and (ch["cell_pairs"] == 0 or precision == capi.SWE_FP32)
    assert ch["queue"] in (0, 1) and (ch["queue"] == 0 or (precision == capi.SWE_FP32 and ch["activity"]))
    assert ch["n_candidates"] >= 20 and 0 < ch["ms_best"] <= ch["ms_before"]
    t_ens = ens.step(90, cfl)
    for k, m in enumerate(meshes):
        assert m.step(103, cfl[k]) == t_ens[k]
        assert _same(ens.get_state(k), m.get_state()), f"member {k}"
    ens.close()
    for m in meshes:
        m.close()


@pytest.mark.parametrize("precision", [capi.SWE_FP64, capi.SWE_FP32])
def test_autotune_choice_survives_set_state_adjoint_style_calls(precision):
    # whichever shape (and activity mode) the tuner keeps, later set_state,
    # boundary changes and frozen-dt steps give the untuned mesh's results
    mi = mg.river(160, 24, seed=6, n_bumps=20)
    tuned, plain = _mesh(mi, precision), _mesh(mi, precision)
    tuned.autotune(trial_steps=2)
    for m in (tuned, plain):
        m.step(20)
        m.set_state(*(x.astype(m.dtype) for x in (mi.h, mi.hu, mi.hv)))
        m.step(31)
        m.set_bc(mi.bcs[1][0], mg.BC_WALL)
        m.step(17)
    if precision == capi.SWE_FP64:
        dts = np.full(9, 0.05)
        assert tuned.step_dt(dts) == plain.step_dt(dts)
    assert tuned.step(40) == plain.step(40)
    assert _same(tuned.get_state(), plain.get_state())
