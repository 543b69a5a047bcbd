"""CPU-side checks of the CUDA library: it loads, exports every symbol the
header declares, and its host preprocessing (Section 3.1 geometry,
neighbours across shared edges, canonical edge orientation, locality order)
agrees with the oracle's independent mesh build.  No GPU is used."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2010_14416_gb300 import build as libbuild
from paper_2010_14416_gb300 import capi
from paper_2010_14416_gb300 import meshgen as mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    return capi.load()


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"SWE_API\s+[\w\s\*]*?\b(swe_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    declared = _declared_symbols()
    assert len(declared) >= 14
    lib = capi.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(capi.EXPORTS)


def test_no_gpu_needed_for_config_default():
    cfg = capi.config_default()
    assert cfg.precision == capi.SWE_FP64 and cfg.g == 9.81 and cfg.h_dry == 1e-6
    assert cfg.reorder == capi.SWE_REORDER_HILBERT


@pytest.mark.parametrize("precision", [capi.SWE_FP64, capi.SWE_FP32])
@pytest.mark.parametrize("reorder", [capi.SWE_REORDER_NONE, capi.SWE_REORDER_RCM,
                                     capi.SWE_REORDER_HILBERT])
def test_preprocess_agrees_with_oracle_geometry(reorder, precision):
    # FP64 meshes number each cell's edges as the caller (and the oracle) do;
    # FP32 meshes may rotate the numbering (the shared edge of a cell pair is
    # local edge 0), keeping the counter-clockwise cycle
    mi = mg.river(60, 12, seed=4, shuffle=True)
    P = capi.mesh_preprocess(mi.nodes, mi.tris, reorder, precision)
    perm = P["perm"]
    n = mi.n_cells
    assert np.array_equal(np.sort(perm), np.arange(n))          # bijection
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    O = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning).geometry()
    # per cell: area, inscribed radius
    assert np.allclose(1.0 / P["inv_area"], O["area"][perm], rtol=1e-13)
    assert np.allclose(P["rin"], O["rin"][perm], rtol=1e-13)
    # per edge: the set of (neighbour, L n) pairs matches the oracle's
    code = P["code"]
    for c in range(0, n, 7):
        o = perm[c]
        lib_edges = []
        for j in range(3):
            k = code[c, j]
            nb = -1 if k < 0 else int(perm[k & 0x3FFFFFFF])
            lib_edges.append((nb, round(P["ln"][c, j, 0], 9), round(P["ln"][c, j, 1], 9)))
            if k >= 0:
                # canonical orientation: flip bit set iff the neighbour has the lower caller index
                assert bool(k & 0x40000000) == (nb < o)
        orc_edges = [(int(O["nbr"][o, j]) if O["nbr"][o, j] >= 0 else -1,
                      round(O["len"][o, j] * O["nx"][o, j], 9), round(O["len"][o, j] * O["ny"][o, j], 9))
                     for j in range(3)]
        if precision == capi.SWE_FP64:
            assert lib_edges == orc_edges
        else:
            assert lib_edges in [orc_edges[r:] + orc_edges[:r] for r in range(3)]


def test_shared_edges_have_bitwise_opposite_normals():
    mi = mg.river(40, 8, seed=2, shuffle=True)
    P = capi.mesh_preprocess(mi.nodes, mi.tris, capi.SWE_REORDER_HILBERT)
    code, ln = P["code"], P["ln"]
    n = mi.n_cells
    for c in range(n):
        for j in range(3):
            k = code[c, j]
            if k < 0:
                continue
            k &= 0x3FFFFFFF
            jj = [q for q in range(3) if code[k, q] >= 0 and (code[k, q] & 0x3FFFFFFF) == c]
            assert len(jj) == 1
            assert ln[k, jj[0], 0] == -ln[c, j, 0] and ln[k, jj[0], 1] == -ln[c, j, 1]


def test_cell_pairs_share_local_edge_zero():
    # the pairing of FP32 mesh preprocessing: for the RCM and Hilbert orders most
    # positions (2p, 2p+1) hold two cells whose local edge 0 is their shared
    # edge, whole warps (32 pairs) are all paired or all unpaired, and every
    # mode numbers a cell's edges alike (same caller neighbour and L n at each
    # local edge)
    mi = mg.river(160, 32, seed=3, shuffle=True)
    n = mi.n_cells
    per_mode = {}
    for r in (capi.SWE_REORDER_NONE, capi.SWE_REORDER_RCM, capi.SWE_REORDER_HILBERT):
        P = capi.mesh_preprocess(mi.nodes, mi.tris, r, capi.SWE_FP32)
        perm, code, ln = P["perm"], P["code"], P["ln"]
        inv = np.empty(n, np.int64)
        inv[perm] = np.arange(n)
        nb = np.where(code >= 0, perm[np.where(code >= 0, code & 0x3FFFFFFF, 0)], -1)   # caller numbering
        per_mode[r] = (nb[inv], ln[inv])
        if r == capi.SWE_REORDER_NONE:
            continue
        a, b = np.arange(0, n - 1, 2), np.arange(1, n, 2)
        shared = (code[a, 0] >= 0) & (code[b, 0] >= 0) & ((code[a, 0] & 0x3FFFFFFF) == b) & \
                 ((code[b, 0] & 0x3FFFFFFF) == a)
        assert shared.mean() > 0.85, (r, shared.mean())
        w = shared[: len(shared) // 32 * 32].reshape(-1, 32).sum(axis=1)
        assert np.mean((w == 0) | (w == 32)) > 0.95, r
    ref_nb, ref_ln = per_mode[capi.SWE_REORDER_NONE]
    for r in (capi.SWE_REORDER_RCM, capi.SWE_REORDER_HILBERT):
        assert np.array_equal(per_mode[r][0], ref_nb)
        assert np.array_equal(per_mode[r][1], ref_ln)


def test_locality_orders_shrink_neighbour_distance():
    mi = mg.river(200, 40, seed=1, shuffle=True)
    spans = {}
    for r in (capi.SWE_REORDER_NONE, capi.SWE_REORDER_RCM, capi.SWE_REORDER_HILBERT):
        code = capi.mesh_preprocess(mi.nodes, mi.tris, r)["code"]
        c = np.repeat(np.arange(mi.n_cells), 3).reshape(-1, 3)
        valid = code >= 0
        d = np.abs((code & 0x3FFFFFFF) - c)[valid]
        spans[r] = np.median(d)
    assert spans[capi.SWE_REORDER_HILBERT] < spans[capi.SWE_REORDER_NONE] / 50
    assert spans[capi.SWE_REORDER_RCM] < spans[capi.SWE_REORDER_NONE] / 50


def test_malformed_meshes_rejected_by_host_preprocessing():
    nodes = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0], [0.5, -1.0]])
    with pytest.raises(capi.SWEError) as e:
        capi.mesh_preprocess(nodes, np.array([[0, 1, 2], [0, 1, 3], [0, 4, 1]]))
    assert e.value.code == capi.SWE_EMESH
    with pytest.raises(capi.SWEError) as e:
        capi.mesh_preprocess(np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0]]), np.array([[0, 1, 2]]))
    assert e.value.code == capi.SWE_EMESH
    with pytest.raises(capi.SWEError) as e:
        capi.mesh_preprocess(nodes, np.array([[0, 1, 9]]))
    assert e.value.code == capi.SWE_EMESH
    with pytest.raises(capi.SWEError) as e:
        capi.mesh_preprocess(nodes, np.zeros((0, 3), np.int32))
    assert e.value.code == capi.SWE_EINVAL


@pytest.mark.parametrize("kw", [dict(g=0.0), dict(g=float("inf")), dict(h_dry=-1e-6), dict(h_dry=float("nan")),
                                dict(h_dry=float("inf")), dict(h_dry=1e-40), dict(precision=7), dict(flux=5), dict(geometry_early=2),
                                dict(activity=3), dict(edge_pass=2), dict(edge_pass=-1), dict(grid=-1), dict(debug_checks=2),
                                dict(activity=1, edge_pass=1),
                                dict(block_size=96)])
def test_invalid_configs_rejected_before_any_device_work(kw):
    # swe_mesh_create validates its configuration before it touches the
    # device, so these fail the same way with or without a GPU
    mi = mg.dam_break_4k()
    with pytest.raises(capi.SWEError) as e:
        capi.Mesh(mi.nodes, mi.tris, mi.z, mi.manning, **kw)
    assert e.value.code == capi.SWE_EINVAL


@pytest.mark.parametrize("field,value", [("manning", -0.01), ("manning", float("inf")), ("manning", float("nan")),
                                         ("z", float("inf")), ("z", float("nan"))])
def test_invalid_fields_rejected_before_any_device_work(field, value):
    mi = mg.dam_break_4k()
    z, manning = mi.z.copy(), mi.manning.copy()
    (manning if field == "manning" else z)[17] = value
    with pytest.raises(capi.SWEError) as e:
        capi.Mesh(mi.nodes, mi.tris, z, manning)
    assert e.value.code == capi.SWE_EINVAL


def test_debug_check_predicate():
    # the check debug_checks applies to each neighbour code before use: an
    # interior code names a cell below n (bit 30 marks the edge's right side),
    # a boundary code -1 - g names a group below n_groups
    ok = capi.debug_code_ok
    n, ng = 1000, 3
    flip = 1 << 30
    assert ok(0, n, ng) and ok(n - 1, n, ng) and ok((n - 1) | flip, n, ng)
    assert not ok(n, n, ng) and not ok(n | flip, n, ng) and not ok((1 << 30) - 1, n, ng)
    assert ok(-1, n, ng) and ok(-ng, n, ng)
    assert not ok(-ng - 1, n, ng) and not ok(-(2 ** 31), n, ng)
    assert not ok(0, 0, ng) and not ok(-1, n, 0)
    # every code of a valid mesh passes, with the mesh's own sizes
    mi = mg.river(30, 6, seed=2)
    P = capi.mesh_preprocess(mi.nodes, mi.tris)
    assert all(ok(int(c), mi.n_cells, 1) for c in P["code"].ravel())
