"""Pins for the oracle's whole-mesh output (Alg. 1 + Alg. 2): exhaustive enumeration with
linear programs, closed-form solids, and the watertightness invariants of Thm. 1."""
import math

import numpy as np
import pytest

from synth import octahedron, polytope_max_of_planes, sphere_net, tiny_net
from tests import pins

RAY = np.array([[1.0, 0.37, 0.21]]) / np.linalg.norm([1.0, 0.37, 0.21])


@pytest.fixture(scope="module")
def sphere_mesh(oracle_mod):
    """The 3-[64]x4-1 geometric-init net, one +x ray (about 4.4e4 faces; ~10 s)."""
    return oracle_mod.mesh_from_rays(sphere_net(), np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]))


# ------------------------------------------------------------------------------------------
# exhaustive enumeration (<= 16 ReLUs)


@pytest.mark.parametrize("widths,seed", [((8, 8), 11), ((6, 5, 4), 12), ((5, 5, 5), 13)])
def test_bruteforce_face_set(oracle_mod, widths, seed):
    mlp = tiny_net(widths, seed)
    brute = pins.enumerate_faces(mlp, oracle_mod.DEFAULT_BOX)
    assert len(brute) > 20
    net = oracle_mod.OracleNet(mlp)
    # seeded from every face found by enumeration: the oracle must find exactly that set
    mesh = oracle_mod.march(net, list(brute.items()))
    assert not mesh.failed and mesh.empty == 0 and mesh.degenerate == 0
    assert set(f.key for f in mesh.faces) == set(brute)
    # seeded from one ray: a subset of it, closed under the neighbour relation
    one = oracle_mod.march(net, oracle_mod.seed_cells(net, np.zeros((1, 3)), RAY))
    keys = set(f.key for f in one.faces)
    assert keys and keys <= set(brute)
    for f in one.faces:
        for e in f.edges:
            if e < mlp.N:
                assert f.key ^ (1 << e) in keys


# ------------------------------------------------------------------------------------------
# closed forms


def test_octahedron_closed_form(oracle_mod):
    # F = |x|_1 - 1: one triangle per orthant sigma with vertices sigma_i e_i; the edge
    # between sigma_a e_a and sigma_b e_b lies on the third coordinate plane, carried by the
    # relu(x_c) neuron c.  CCW from +grad F = sigma; canonical start at the vertex on the
    # planes (0, 1), i.e. sigma_z e_z.
    net, mesh = oracle_mod.mesh_from_rays(octahedron(), np.zeros((1, 3)), RAY)
    assert len(mesh.faces) == 8 and not mesh.failed and mesh.degenerate == 0
    got = mesh.by_key()
    for sx in (1, -1):
        for sy in (1, -1):
            for sz in (1, -1):
                key = (sx > 0) | (sy > 0) << 1 | (sz > 0) << 2 | 0b111000
                f = got[key]
                if sx * sy * sz > 0:
                    V = [[0, 0, sz], [sx, 0, 0], [0, sy, 0]]; E = [1, 2, 0]
                else:
                    V = [[0, 0, sz], [0, sy, 0], [sx, 0, 0]]; E = [0, 2, 1]
                assert f.edges == E
                np.testing.assert_allclose(f.verts, V, rtol=0, atol=1e-15)
                assert abs(f.area() - math.sqrt(3) / 2) < 1e-14
    xyz, faces, _ = mesh.assemble()
    assert len(xyz) == 6 and pins.euler_characteristic(len(xyz), faces) == 2
    assert abs(pins.signed_volume(xyz, faces) - 4.0 / 3.0) < 1e-14


def test_polytope_closed_form(oracle_mod):
    mlp = polytope_max_of_planes()
    normals, offset = mlp.meta["normals"], mlp.meta["offset"]
    area_ref, vol_ref, Vref = pins.polytope_facets(normals, offset)
    net, mesh = oracle_mod.mesh_from_rays(mlp, np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]))
    assert not mesh.failed and mesh.degenerate == 0 and mesh.open_faces() == 0
    area = np.zeros(12)
    for f in mesh.faces:
        n = f.aF[:3] / np.linalg.norm(f.aF[:3])
        i = int(np.argmax(normals @ n))
        assert normals[i] @ n > 1 - 1e-12                       # face lies on facet plane i
        assert abs(f.aF[3] / np.linalg.norm(f.aF[:3]) + offset) < 1e-12
        area[i] += f.area()
    np.testing.assert_allclose(area, area_ref, rtol=1e-10, atol=1e-12)
    xyz, faces, _ = mesh.assemble()
    assert abs(pins.signed_volume(xyz, faces) - vol_ref) < 1e-10 * vol_ref
    for v in Vref:                                              # every polytope corner is a mesh vertex
        assert np.min(np.linalg.norm(xyz - v, axis=1)) < 1e-10
    assert pins.euler_characteristic(len(xyz), faces) == 2


# ------------------------------------------------------------------------------------------
# invariants (Thm. 1 and Eq. 12)


def _check_invariants(net, mesh, closed, chi=None):
    N = net.N
    by = mesh.by_key()
    # each edge (cell, neuron) has its reciprocal (cell ^ e_k, neuron)
    for f in mesh.faces:
        for e in f.edges:
            if e < N:
                g = by.get(f.key ^ (1 << e))
                assert g is not None and e in g.edges
    xyz, faces, vkeys = mesh.assemble()
    E = pins.mesh_edges(faces)
    for (a, b), fl in E.items():
        if closed:
            assert len(fl) == 2
        else:
            assert len(fl) in (1, 2)
    if closed:
        use = np.bincount(np.concatenate([np.asarray(f) for f in faces]), minlength=len(xyz))
        assert use.min() >= 3
        assert mesh.open_faces() == 0
    if chi is not None:
        assert pins.euler_characteristic(len(xyz), faces) == chi
    # vertices on the zero set; every face inside its own cell
    rng = np.random.default_rng(0)
    idx = rng.choice(len(xyz), min(len(xyz), 3000), replace=False)
    for v in xyz[idx]:
        assert abs(net.F(v)) <= 1e-9
    for fi in rng.choice(len(mesh.faces), min(len(mesh.faces), 2000), replace=False):
        f = mesh.faces[fi]
        c = f.verts.mean(0)
        assert np.array_equal(net.state(c), net_state_of(f.key, N))


def net_state_of(key, N):
    return np.array([(key >> k) & 1 for k in range(N)], dtype=np.uint8)


def test_invariants_small(oracle_mod):
    for mlp, ray, closed, chi in [(octahedron(), RAY, True, 2),
                                  (polytope_max_of_planes(), RAY, True, 2),
                                  (tiny_net((8, 8), 11), RAY, False, None)]:
        net, mesh = oracle_mod.mesh_from_rays(mlp, np.zeros((1, 3)), ray)
        assert not mesh.failed
        _check_invariants(net, mesh, closed, chi)


def test_invariants_sphere_net(oracle_mod, sphere_mesh):
    net, mesh = sphere_mesh
    assert len(mesh.faces) > 10000 and not mesh.failed and mesh.degenerate == 0
    _check_invariants(net, mesh, closed=True, chi=2)


def test_face_area_of_a_tiny_face_far_from_the_origin(oracle_mod):
    # A face whose sides (3.4e-9) are long next to delta but tiny next to its distance from the
    # origin: its area (closed form 1/2 |a x b|, here 5e-18) must survive, far above the 1e-24 B^2
    # threshold below which a face is dropped as empty.  Summing V_i x V_{i+1} on the absolute
    # coordinates cancels to 0 in FP64; about the first vertex it keeps the closed form.
    p0 = np.array([0.7, -1.1, 0.9])
    a = np.array([3.3e-9, 0.4e-9, -0.2e-9])
    b = np.array([-0.6e-9, 3.1e-9, 1.1e-9])
    V = np.stack([p0, p0 + a, p0 + b])
    exact = 0.5 * np.linalg.norm(np.cross(a, b))
    f = oracle_mod.Face(key=0, edges=[0, 1, 2], verts=V, aF=np.array([0.0, 0.0, 1.0, 0.0]))
    assert abs(f.area() - exact) <= 1e-6 * exact, (f.area(), exact)
    assert f.area() > 1e-24 * 1.5 ** 2
    # and the orientation test sees the same normal as the closed form
    nrm = oracle_mod.newell(V)
    assert np.dot(nrm, np.cross(a, b)) > 0.0
