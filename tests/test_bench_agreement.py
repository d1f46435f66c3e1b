"""The bench's comparison of its headline mesh with the oracle's (exactness.vs_oracle), checked
on the CPU: an oracle mesh packed in the GPU mesh layout agrees with itself exactly, and a
perturbed vertex, a changed edge cycle or a missing face is reported."""
import types

import numpy as np
import pytest

from synth import tiny_net

RAY = np.array([[1.0, 0.37, 0.21]]) / np.linalg.norm([1.0, 0.37, 0.21])


def _packed(ref, N):
    xyz, fv, ep, off, keys = [], [], [], [0], []
    kw = (N + 63) // 64
    for f in ref.faces:
        for j, e in enumerate(f.edges):
            fv.append(len(xyz))
            xyz.append(f.verts[j])
            ep.append(e)
        off.append(len(fv))
        keys.append([(f.key >> (64 * w)) & ((1 << 64) - 1) for w in range(kw)])
    return types.SimpleNamespace(n_faces=len(ref.faces), face_offsets=np.array(off), face_vertices=np.array(fv),
                                 edge_planes=np.array(ep), face_keys=np.array(keys, dtype=np.uint64),
                                 xyz=np.array(xyz))


@pytest.fixture(scope="module")
def case(oracle_mod):
    mlp = tiny_net((6, 5, 4), 12)
    net, ref = oracle_mod.mesh_from_rays(mlp, np.zeros((1, 3)), RAY)
    return mlp, ref


def test_identical_mesh(case):
    import bench
    mlp, ref = case
    r = bench.oracle_agreement(ref, _packed(ref, mlp.N))
    assert r["whole_mesh_identical"] and r["max_rel_vertex_err"] == 0.0 and r["oracle_faces"] == len(ref.faces)


def test_differences_are_reported(case):
    import bench
    mlp, ref = case
    mesh = _packed(ref, mlp.N)
    mesh.xyz = mesh.xyz + 1e-7
    r = bench.oracle_agreement(ref, mesh)
    assert 1e-7 < r["max_rel_vertex_err"] < 1e-6 and r["whole_mesh_identical"]
    mesh = _packed(ref, mlp.N)
    o = mesh.face_offsets
    e = mesh.edge_planes
    e[o[0]], e[o[0] + 1] = e[o[0] + 1], e[o[0]]                                 # another cycle
    assert bench.oracle_agreement(ref, mesh)["edge_cycles_differing"] >= 1
    mesh = _packed(ref, mlp.N)
    mesh.face_keys[0] ^= np.uint64(1 << 40)                                     # a face the oracle lacks
    r = bench.oracle_agreement(ref, mesh)
    assert r["missing_in_gpu"] == 1 and not r["whole_mesh_identical"]
