"""Host post-processing of a copied-out mesh (am_mesh_canonicalize, am_mesh_triangulate): pure
host logic in the C library, exercised on CPU on meshes the oracle assembles.  The canonical
form is rebuilt independently here (Python sort of the keys, first-appearance numbering), and
the fan triangulation is pinned by the polytope's closed-form volume and Euler characteristic."""
import numpy as np
import pytest

from synth import polytope_max_of_planes, sphere_net, tiny_net
from tests import pins

RAY = np.array([[1.0, 0.37, 0.21]]) / np.linalg.norm([1.0, 0.37, 0.21])


@pytest.fixture(scope="module")
def am():
    from paper_2106_10031_gb300 import build
    build.build()
    import paper_2106_10031_gb300 as am_mod
    return am_mod


def _library_mesh(am, oracle_mod, mlp, dirs=RAY):
    """The oracle's assembled mesh in the library's array layout."""
    net, ref = oracle_mod.mesh_from_rays(mlp, np.zeros((len(dirs), 3)), dirs)
    xyz, faces, _ = ref.assemble()
    kw = (mlp.N + 63) // 64
    off = np.zeros(len(faces) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(f) for f in faces])
    fv = np.concatenate([np.asarray(f, dtype=np.int32) for f in faces])
    fe = np.concatenate([np.asarray(f.edges, dtype=np.int32) for f in ref.faces])
    keys = np.stack([oracle_mod.key_to_words(f.key, kw) for f in ref.faces]).astype(np.uint64)
    return am.Mesh(np.asarray(xyz, dtype=np.float64), off, fv, fe, keys, ref.open_faces()), ref


def _shuffled(am, mesh, seed):
    """Same surface, other order: faces permuted, rings rotated, vertex ids permuted."""
    rng = np.random.default_rng(seed)
    F, V = mesh.n_faces, len(mesh.xyz)
    perm_v = rng.permutation(V)                      # old id -> new id
    xyz = np.empty_like(mesh.xyz)
    xyz[perm_v] = mesh.xyz
    order = rng.permutation(F)
    fv, fe, off = [], [], [0]
    for f in order:
        a, b = mesh.face_offsets[f], mesh.face_offsets[f + 1]
        r = int(rng.integers(0, b - a))
        fv.append(np.roll(perm_v[mesh.face_vertices[a:b]], -r))
        fe.append(np.roll(mesh.edge_planes[a:b], -r))
        off.append(off[-1] + b - a)
    return am.Mesh(xyz, np.asarray(off, dtype=np.int64), np.concatenate(fv).astype(np.int32),
                   np.concatenate(fe).astype(np.int32), mesh.face_keys[order].copy(), mesh.n_open_faces)


def _expected_canonical(mesh):
    """The canonical form, written out in Python."""
    kint = [int.from_bytes(mesh.face_keys[i].tobytes(), "little") for i in range(mesh.n_faces)]
    order = sorted(range(mesh.n_faces), key=lambda i: kint[i])
    fv, fe, off = [], [], [0]
    for f in order:
        a, b = mesh.face_offsets[f], mesh.face_offsets[f + 1]
        e, v = list(mesh.edge_planes[a:b]), list(mesh.face_vertices[a:b])
        m = len(e)
        pairs = [(min(e[j - 1], e[j]), max(e[j - 1], e[j])) for j in range(m)]
        j0 = min(range(m), key=lambda j: pairs[j])
        fv += v[j0:] + v[:j0]
        fe += e[j0:] + e[:j0]
        off.append(off[-1] + m)
    new = {}
    for v in fv:
        new.setdefault(v, len(new))
    xyz = np.empty_like(mesh.xyz)
    for old, nid in new.items():
        xyz[nid] = mesh.xyz[old]
    return (xyz, np.asarray(off), np.asarray([new[v] for v in fv]), np.asarray(fe),
            mesh.face_keys[order])


def _assert_same(m, xyz, off, fv, fe, keys):
    assert np.array_equal(m.xyz, xyz)
    assert np.array_equal(m.face_offsets, off)
    assert np.array_equal(m.face_vertices, fv)
    assert np.array_equal(m.edge_planes, fe)
    assert np.array_equal(m.face_keys, keys)


@pytest.mark.parametrize("make", [polytope_max_of_planes, lambda: tiny_net((6, 5, 4), 12),
                                  lambda: sphere_net(seed=21, width=32, depth=4, sigma=0.05)])
def test_canonical_form_is_the_definition_and_order_free(am, oracle_mod, make):
    mesh, _ = _library_mesh(am, oracle_mod, make())
    want = _expected_canonical(mesh)
    _assert_same(am.canonicalize(mesh), *want)
    for seed in (1, 2):
        got = am.canonicalize(_shuffled(am, mesh, seed))
        _assert_same(got, *want)
        assert got.n_open_faces == mesh.n_open_faces


def test_canonical_form_of_a_multi_word_key(am, oracle_mod):
    # N = 128: two key words, the most significant one decides first
    mlp = sphere_net(seed=21, width=32, depth=4, sigma=0.05)
    mesh, _ = _library_mesh(am, oracle_mod, mlp)
    assert mesh.face_keys.shape[1] == 2
    got = am.canonicalize(_shuffled(am, mesh, 3))
    k = [int.from_bytes(got.face_keys[i].tobytes(), "little") for i in range(got.n_faces)]
    assert k == sorted(k)


def test_fan_triangulation_of_the_polytope(am, oracle_mod):
    mlp = polytope_max_of_planes()
    mesh, ref = _library_mesh(am, oracle_mod, mlp)
    tri = am.triangulate(mesh)
    assert tri.shape == (len(mesh.face_vertices) - 2 * mesh.n_faces, 3)
    area_ref, vol_ref, _ = pins.polytope_facets(mlp.meta["normals"], mlp.meta["offset"])
    assert abs(pins.signed_volume(mesh.xyz, tri.tolist()) - vol_ref) < 1e-9
    assert pins.euler_characteristic(len(mesh.xyz), tri.tolist()) == 2
    a = 0.5 * np.linalg.norm(np.cross(mesh.xyz[tri[:, 1]] - mesh.xyz[tri[:, 0]],
                                      mesh.xyz[tri[:, 2]] - mesh.xyz[tri[:, 0]]), axis=1).sum()
    assert abs(a - area_ref.sum()) < 1e-9
    # every triangle keeps its face's orientation (normal along +grad F = a_F[0:3])
    fid = np.repeat(np.arange(mesh.n_faces), np.diff(mesh.face_offsets) - 2)
    n = np.cross(mesh.xyz[tri[:, 1]] - mesh.xyz[tri[:, 0]], mesh.xyz[tri[:, 2]] - mesh.xyz[tri[:, 0]])
    aF = np.stack([ref.faces[i].aF[:3] for i in fid])
    assert np.all(np.einsum("ij,ij->i", n, aF) > 0)


def test_inconsistent_arrays_are_refused(am, oracle_mod):
    mesh, _ = _library_mesh(am, oracle_mod, polytope_max_of_planes())
    bad = _shuffled(am, mesh, 4)
    bad.face_vertices[0] = len(bad.xyz)                      # a vertex index out of range
    with pytest.raises(am.AMError) as e:
        am.canonicalize(bad)
    assert e.value.status == 1
    bad = _shuffled(am, mesh, 4)
    bad.face_offsets[1] = bad.face_offsets[0] + 2            # a face with two corners
    with pytest.raises(am.AMError):
        am.triangulate(bad)
    bad = _shuffled(am, mesh, 4)
    bad.edge_planes = bad.edge_planes[:-1]                    # arrays of inconsistent lengths
    with pytest.raises(ValueError):
        am.canonicalize(bad)
