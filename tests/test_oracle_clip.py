"""Pins for the oracle's face clip: Alg. 2 (pivoting) against Alg. 1 (all pairs, a second
independent implementation in numpy) and against Qhull's half-space intersection."""
import numpy as np
import pytest

from synth import octahedron, polytope_max_of_planes, sphere_net, tiny_net
from tests import pins


def _match(V1, V2, tol):
    assert len(V1) == len(V2), (len(V1), len(V2))
    for v in V1:
        d = np.min(np.linalg.norm(V2 - v, axis=1))
        assert d <= tol, d


def _cells(oracle_mod, mlp, max_cells):
    net = oracle_mod.OracleNet(mlp)
    d = np.array([[1.0, 0.37, 0.21]])
    seeds = oracle_mod.seed_cells(net, np.zeros((1, 3)), d / np.linalg.norm(d))
    mesh = oracle_mod.march(net, seeds, max_cells=max_cells)
    assert not mesh.failed and mesh.faces
    return net, mesh


@pytest.mark.parametrize("make,max_cells", [
    (octahedron, None), (polytope_max_of_planes, None), (lambda: tiny_net((6, 5, 4), 12), None),
    (sphere_net, 40),
])
def test_pivot_equals_allpairs_and_qhull(oracle_mod, make, max_cells):
    net, mesh = _cells(oracle_mod, make(), max_cells)
    for f in mesh.faces:
        C, aF = net.cell_rows(oracle_mod.key_to_state(f.key, net.N))
        V2, P2 = oracle_mod.face_allpairs(C, aF)
        _match(f.verts, V2, 1e-9)
        # same cyclic sequence of defining plane pairs
        pairs1 = [f.vertex_pair(i) for i in range(len(f.edges))]
        pairs2 = [tuple(sorted(map(int, p))) for p in P2]
        assert sorted(pairs1) == sorted(pairs2)
        V3 = pins.halfspace_polygon(C, aF, f.verts.mean(0), oracle_mod.DEFAULT_BOX)
        _match(f.verts, V3, 1e-8)
        # orientation: CCW seen from +grad F
        assert oracle_mod.newell(f.verts) @ aF[:3] > 0


def test_consecutive_edges_share_the_vertex(oracle_mod):
    net, mesh = _cells(oracle_mod, sphere_net(), 60)
    for f in mesh.faces:
        C, aF = net.cell_rows(oracle_mod.key_to_state(f.key, net.N))
        m = len(f.edges)
        for i in range(m):
            a, b = f.edges[i - 1], f.edges[i]
            v = f.verts[i]
            for p in (a, b):
                r = C[p]
                assert abs(r[:3] @ v + r[3]) <= 1e-12 * (1 + np.abs(r).sum())
            assert abs(aF[:3] @ v + aF[3]) <= 1e-12 * (1 + np.abs(aF).sum())


def test_seed_point_lies_on_face_inside_cell(oracle_mod):
    for mlp in (sphere_net(), tiny_net((8, 8), 11), polytope_max_of_planes()):
        net = oracle_mod.OracleNet(mlp)
        rc, x, s, it = net.seed_ray(np.zeros(3), np.array([1.0, 0.0, 0.0]))
        assert rc == 0
        pre, F = net.forward(x)
        assert abs(F) < 1e-12
        assert np.array_equal((pre > 0).astype(np.uint8), s)


def test_seed_ray_without_sign_change_is_an_error(oracle_mod):
    net = oracle_mod.OracleNet(sphere_net())
    rc, *_ = net.seed_ray(np.zeros(3), np.array([1.0, 0.0, 0.0]), R=0.05)
    assert rc == -4
