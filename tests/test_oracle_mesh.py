"""Pins for the oracle's mesh geometry (Section 3.1, Eq 9; Eq 15's inscribed
radius; neighbours across shared edges, Section 4.2) against invariants and
hand-computed values."""
import math

import numpy as np
import pytest

import oracle
from paper_2010_14416_gb300 import meshgen as mg


def _mesh(mi):
    return oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)


def test_unit_right_triangle():
    nodes = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    tris = np.array([[0, 1, 2]], np.int32)
    M = oracle.Mesh(nodes, tris, [0.0], [0.0])
    geo = M.geometry()
    assert geo["area"][0] == 0.5
    assert geo["rin"][0] == pytest.approx((2 - math.sqrt(2)) / 2, abs=1e-15)
    assert geo["rin"][0] == pytest.approx(0.292893218813, abs=1e-12)
    # edges (0,1), (1,2), (2,0): outward normals (0,-1), (1,1)/sqrt2, (-1,0)
    assert np.allclose(geo["nx"][0], [0.0, 1 / math.sqrt(2), -1.0], atol=1e-15)
    assert np.allclose(geo["ny"][0], [-1.0, 1 / math.sqrt(2), 0.0], atol=1e-15)
    assert np.allclose(geo["len"][0], [1.0, math.sqrt(2), 1.0], atol=1e-15)
    assert np.all(geo["nbr"][0] == -1)


def test_clockwise_input_is_reoriented():
    nodes = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    a = oracle.Mesh(nodes, np.array([[0, 1, 2]], np.int32), [0.0], [0.0]).geometry()
    b = oracle.Mesh(nodes, np.array([[0, 2, 1]], np.int32), [0.0], [0.0]).geometry()
    assert a["area"][0] == b["area"][0] and a["rin"][0] == b["rin"][0]
    # same set of outward normals
    sa = sorted(zip(np.round(a["nx"][0], 14), np.round(a["ny"][0], 14)))
    sb = sorted(zip(np.round(b["nx"][0], 14), np.round(b["ny"][0], 14)))
    assert sa == sb


@pytest.mark.parametrize("maker", [lambda: mg.canal(40, 4, 200.0, 10.0, 0.2, 5),
                                   lambda: mg.river(60, 12, seed=3)])
def test_geometry_invariants(maker):
    mi = maker()
    M = _mesh(mi)
    geo = M.geometry()
    Lx, Ly = mi.meta["Lx"], mi.meta["Ly"]
    assert geo["area"].sum() == pytest.approx(Lx * Ly, rel=1e-12)
    # closed triangle: sum_j L_ij n_ij = 0
    sx = (geo["len"] * geo["nx"]).sum(axis=1)
    sy = (geo["len"] * geo["ny"]).sum(axis=1)
    scale = geo["len"].max()
    assert np.abs(sx).max() < 1e-12 * scale and np.abs(sy).max() < 1e-12 * scale
    # unit normals
    assert np.allclose(geo["nx"] ** 2 + geo["ny"] ** 2, 1.0, atol=1e-14)
    # neighbour symmetry with opposite normals and equal lengths
    nbr = geo["nbr"]
    n = mi.n_cells
    for i in range(n):
        for j in range(3):
            k = nbr[i, j]
            if k < 0:
                continue
            jj = np.where(nbr[k] == i)[0]
            assert jj.size == 1
            jj = jj[0]
            assert geo["len"][k, jj] == pytest.approx(geo["len"][i, j], rel=1e-14)
            assert geo["nx"][k, jj] == pytest.approx(-geo["nx"][i, j], abs=1e-14)
            assert geo["ny"][k, jj] == pytest.approx(-geo["ny"][i, j], abs=1e-14)
    nx_, ny_ = mi.meta["nx"], mi.meta["ny"]
    assert (nbr < 0).sum() == 2 * (nx_ + ny_)
    # inscribed radius: 2A / perimeter, and no larger than any altitude / 2
    assert np.allclose(geo["rin"], 2 * geo["area"] / geo["len"].sum(axis=1), rtol=1e-14)


def test_malformed_meshes_are_rejected():
    nodes = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0], [0.5, -1.0]])
    with pytest.raises(oracle.OracleError):  # three triangles on edge (0,1)
        oracle.Mesh(nodes, np.array([[0, 1, 2], [0, 1, 3], [0, 4, 1]], np.int32),
                    np.zeros(3), np.zeros(3))
    with pytest.raises(oracle.OracleError):  # zero area
        oracle.Mesh(np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0]]),
                    np.array([[0, 1, 2]], np.int32), [0.0], [0.0])
    with pytest.raises(oracle.OracleError):  # index out of range
        oracle.Mesh(nodes, np.array([[0, 1, 7]], np.int32), [0.0], [0.0])


def test_bc_groups_cover_requested_edges():
    mi = mg.river(40, 8, seed=1)
    M = _mesh(mi)
    for pairs, kind, value in mi.bcs:
        M.set_bc(pairs, kind, value)
    nbr = M.geometry()["nbr"]
    assert (nbr == -2).sum() == mi.bcs[0][0].shape[0]   # inflow group 1
    assert (nbr == -3).sum() == mi.bcs[1][0].shape[0]   # stage group 2
    with pytest.raises(oracle.OracleError):
        M.set_bc(np.array([[0, 0]], np.int32), oracle.BC_WALL)
