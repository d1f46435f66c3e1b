"""The bench's comparison of its headline mesh with the oracle's (exactness.vs_oracle), checked
on the CPU: the oracle's own mesh, in the GPU mesh layout, agrees with the oracle (whole-mesh
digest identical, sampled faces re-solved alike), and a perturbed vertex, a changed edge cycle
or a missing face is reported."""
import copy

import numpy as np
import pytest

from synth import tiny_net
from tests import meshcheck

RAY = np.array([[1.0, 0.37, 0.21]]) / np.linalg.norm([1.0, 0.37, 0.21])


@pytest.fixture(scope="module")
def case(oracle_mod):
    mlp = tiny_net((6, 5, 4), 12)
    net, ref = oracle_mod.mesh_from_rays(mlp, np.zeros((1, 3)), RAY)
    am = meshcheck.ArrayMesh(ref, mlp.N)
    return mlp, am, {"digest": meshcheck.digest(am, mlp.N)}


def test_identical_mesh(case):
    import bench
    mlp, am, golden = case
    r = bench.oracle_agreement(mlp, am, golden=golden, sample=50)
    assert r["whole_mesh_identical"] and r["closed"] is True and r["oracle_faces"] == am.n_faces
    assert r["sampled_edge_cycles_differing"] == 0 and r["max_rel_vertex_err"] < 1e-12


def test_differences_are_reported(case):
    import bench
    mlp, am, golden = case
    mesh = copy.deepcopy(am)
    mesh.xyz = mesh.xyz + 1e-7
    r = bench.oracle_agreement(mlp, mesh, golden=golden, sample=50)
    assert 1e-8 < r["max_rel_vertex_err"] < 1e-6 and r["whole_mesh_identical"]
    mesh = copy.deepcopy(am)
    o, e = mesh.face_offsets, mesh.edge_planes
    for f in range(mesh.n_faces):                                               # another cycle everywhere
        e[o[f]], e[o[f] + 1] = e[o[f] + 1], e[o[f]]
    r = bench.oracle_agreement(mlp, mesh, golden=golden, sample=50)
    assert r["sampled_edge_cycles_differing"] >= 1 and not r["whole_mesh_identical"]
    mesh = copy.deepcopy(am)
    mesh.face_keys[0] ^= np.uint64(1 << 3)                                     # a face the oracle lacks
    r = bench.oracle_agreement(mlp, mesh, golden=golden, sample=50)
    assert not r["whole_mesh_identical"] and r["closed"] is not True
