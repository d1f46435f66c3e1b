"""The whole-mesh checks used at full size (tests/meshcheck.py), on the oracle's own meshes:
they accept them, and each catches a planted mistake of the kind it exists for."""
import copy

import numpy as np
import pytest

from synth import polytope_max_of_planes, sphere_net
from tests import meshcheck as mc

X_RAY = np.array([[1.0, 0.0, 0.0]])


@pytest.fixture(scope="module")
def meshes(oracle_mod):
    out = {}
    for mlp in (polytope_max_of_planes(), sphere_net(seed=21, width=32, depth=4)):
        _, ref = oracle_mod.mesh_from_rays(mlp, np.zeros((1, 3)), X_RAY)
        out[mlp.name] = (mlp, mc.ArrayMesh(ref, mlp.N))
    return out


def test_accepts_the_oracle_meshes(meshes):
    mlp, am = meshes["polytope12"]
    assert mc.closure(am, mlp.N)["box_edges"] == 0
    assert mc.vertex_bijection(am, mlp.N) == len(am.xyz)
    d = mc.digest(am, mlp.N)
    assert d["euler"] == 2 and d["open_faces"] == 0          # a convex polytope is a sphere
    mlp, am = meshes["sphere_w32_d4_s21"]
    mc.closure(am, mlp.N)
    assert mc.vertex_bijection(am, mlp.N) == len(am.xyz)


def test_digest_is_order_independent(meshes):
    mlp, am = meshes["sphere_w32_d4_s21"]
    perm = np.random.default_rng(3).permutation(am.n_faces)
    sh = copy.deepcopy(am)
    o = am.face_offsets
    sizes = np.diff(o)[perm]
    sh.face_offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    sh.edge_planes = np.concatenate([np.roll(am.edge_planes[o[f]:o[f + 1]], 2) for f in perm]).astype(np.int32)
    sh.face_vertices = np.concatenate([np.roll(am.face_vertices[o[f]:o[f + 1]], 2) for f in perm]).astype(np.int32)
    sh.face_keys = am.face_keys[perm]
    assert mc.digest(sh, mlp.N) == mc.digest(am, mlp.N)
    assert [len(x) for x in mc.face_diff(am, sh)] == [0, 0, 0, 0]


@pytest.mark.parametrize("mistake", ["flip_key_bit", "drop_face", "reverse_cycle", "merge_vertices",
                                     "split_vertex", "repeat_plane"])
def test_catches_planted_mistakes(meshes, mistake):
    mlp, am = meshes["polytope12"]
    bad = copy.deepcopy(am)
    o = am.face_offsets
    if mistake == "flip_key_bit":
        bad.face_keys[5, 0] ^= np.uint64(1 << 3)
    elif mistake == "drop_face":
        keep = np.arange(am.n_faces) != 7
        sizes = np.diff(o)[keep]
        bad.face_keys = am.face_keys[keep]
        sel = np.concatenate([np.arange(o[f], o[f + 1]) for f in np.flatnonzero(keep)])
        bad.edge_planes, bad.face_vertices = am.edge_planes[sel], am.face_vertices[sel]
        bad.face_offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    elif mistake == "reverse_cycle":
        bad.edge_planes[o[3]:o[4]] = am.edge_planes[o[3]:o[4]][::-1]
    elif mistake == "merge_vertices":
        bad.face_vertices[bad.face_vertices == 7] = 8
    elif mistake == "split_vertex":
        i = np.flatnonzero(am.face_vertices == 7)[0]
        bad.face_vertices[i] = len(am.xyz) - 1
    elif mistake == "repeat_plane":
        # a zero-length edge: one plane pair listed twice in a face (the defect of a bad clip)
        f = 3
        ring = list(am.edge_planes[o[f]:o[f + 1]])
        ring = ring + ring[:2]
        sizes = np.diff(o).copy()
        sizes[f] += 2
        bad.edge_planes = np.concatenate([am.edge_planes[:o[f]], ring, am.edge_planes[o[f + 1]:]]).astype(np.int32)
        fvs = list(am.face_vertices[o[f]:o[f + 1]])
        bad.face_vertices = np.concatenate([am.face_vertices[:o[f]], fvs + fvs[:2],
                                            am.face_vertices[o[f + 1]:]]).astype(np.int32)
        bad.face_offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    caught = False
    for check in (lambda: mc.closure(bad, mlp.N), lambda: mc.vertex_bijection(bad, mlp.N)):
        try:
            check()
        except AssertionError:
            caught = True
    assert caught, f"{mistake} passed the closure and vertex checks"
    if mistake not in ("merge_vertices", "split_vertex"):     # the digest names keys and cycles only
        assert mc.digest(bad, mlp.N) != mc.digest(am, mlp.N)
