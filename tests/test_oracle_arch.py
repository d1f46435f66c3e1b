"""Pins of the oracle for the Sec. 5 architectures (oracle/arch.py): residual blocks of both
kinds (Sec. 5.1) and a final max pooling over sub-networks (Sec. 5.2).  CPU only.

Independent routes: the forward pass by torch (library routine) and torch autograd for the
gradient; a subcell's affine maps by evaluating the network with its states frozen at the
four points 0, e_x, e_y, e_z (the definition of an affine map); the set of non-empty faces by
linear programs over every (pattern, pooled index) of tiny networks (scipy HiGHS); face
polygons by Qhull; and a closed form: the max of two max-of-planes nets is the intersection
of two convex polytopes, whose facet areas and volume Qhull gives from the planes alone."""
import numpy as np
import pytest

from synth import polytope_max_of_planes
from tests import pins


@pytest.fixture(scope="module")
def arch(oracle_mod):
    from oracle import arch as A
    return A


def _resnet(A, seed, first=4, mid=4, with_id=True, with_v=True, depth=3):
    """3 -> first -> mid (-> mid) -> 1, F(0) = -0.5.  depth 3: a second-kind block (V from x)
    ends at layer 2 and a first-kind block (identity from h_1; first == mid) at layer 3.
    depth 2: one block ending at layer 2, first kind (identity from h_1) when with_id, else
    second kind (V from x)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(size=(first, 3))
    W1 /= np.linalg.norm(W1, axis=1, keepdims=True)
    W = [W1] + [0.5 * rng.normal(size=(mid, first if l == 0 else mid)) for l in range(depth - 1)]
    b = [np.zeros(first)] + [0.1 * rng.normal(size=mid) for _ in range(depth - 1)]
    sc = {}
    if depth == 3:
        if with_v:
            sc[2] = (0, rng.normal(size=(mid, 3)))
        if with_id:
            sc[3] = (1, None)
    elif with_id:
        sc[2] = (1, None)
    elif with_v:
        sc[2] = (0, rng.normal(size=(mid, 3)))
    net = A.ResNet(W, b, np.abs(rng.normal(size=mid)) + 0.2, 0.0, sc)
    net.b_out = -0.5 - A.res_forward(net, np.zeros(3))[1]
    return net


def _from_mlp(A, mlp):
    return A.ResNet([np.asarray(W) for W in mlp.weights], [np.asarray(b) for b in mlp.biases],
                    np.asarray(mlp.w_out), float(mlp.b_out), {})


def _torch_F(net, X):
    """Pre-activations and F by torch, from the layer equations; X (P, 3)."""
    import torch
    import torch.nn.functional as tf
    if not isinstance(X, torch.Tensor):
        X = torch.as_tensor(np.atleast_2d(X), dtype=torch.float64)
    hs, pres = [X], []
    for l, (W, b) in enumerate(zip(net.weights, net.biases), start=1):
        a = tf.linear(hs[-1], torch.as_tensor(W), torch.as_tensor(b))
        if l in net.shortcuts:
            src, S = net.shortcuts[l]
            a = a + (hs[src] if S is None else tf.linear(hs[src], torch.as_tensor(S)))
        pres.append(a)
        hs.append(tf.leaky_relu(a, net.slope) if net.slope else torch.relu(a))
    return torch.cat(pres, 1), hs[-1] @ torch.as_tensor(net.w_out) + net.b_out


def _frozen_maps(net, s):
    """Affine rows of every unit and of F with the states frozen to s, from values at 0 and e_i."""
    P = np.vstack([np.zeros(3), np.eye(3)])
    hs, pres, off = [P], [], 0
    for l, (W, b) in enumerate(zip(net.weights, net.biases), start=1):
        a = hs[-1] @ W.T + b
        if l in net.shortcuts:
            src, S = net.shortcuts[l]
            a = a + (hs[src] if S is None else hs[src] @ S.T)
        pres.append(a)
        n = W.shape[0]
        st = np.asarray(s[off:off + n], dtype=np.float64)
        hs.append(a * (st + net.slope * (1.0 - st))[None, :])
        off += n
    pre = np.hstack(pres)
    F = hs[-1] @ net.w_out + net.b_out
    A_ = np.zeros((pre.shape[1], 4))
    A_[:, 3], A_[:, :3] = pre[0], (pre[1:] - pre[0]).T
    return A_, np.array([F[1] - F[0], F[2] - F[0], F[3] - F[0], F[0]])


def test_forward_is_torchs(arch):
    for seed in range(4):
        net = _resnet(arch, seed)
        X = np.random.default_rng(seed).uniform(-1.2, 1.2, size=(20, 3))
        pre_t, F_t = _torch_F(net, X)
        for x, p, f in zip(X, pre_t.detach().numpy(), F_t.detach().numpy()):
            pre, F = arch.res_forward(net, x)
            np.testing.assert_allclose(pre, p, rtol=0, atol=1e-13)
            assert abs(F - f) < 1e-13


@pytest.mark.parametrize("kinds", [(True, True), (True, False), (False, True)])
def test_compose_is_the_frozen_network(arch, kinds):
    for seed in range(3):
        net = _resnet(arch, seed, with_id=kinds[0], with_v=kinds[1])
        rng = np.random.default_rng(100 + seed)
        for _ in range(8):
            s = rng.integers(0, 2, net.N).astype(np.uint8)
            A, aF = arch.res_compose(net, s)
            A2, aF2 = _frozen_maps(net, s)
            np.testing.assert_allclose(A, A2, rtol=0, atol=1e-12)
            np.testing.assert_allclose(aF, aF2, rtol=0, atol=1e-12)


def test_cell_maps_give_F_and_its_gradient(arch):
    import torch
    net = _resnet(arch, 7)
    for x in np.random.default_rng(8).uniform(-1.0, 1.0, size=(25, 3)):
        pre, F = arch.res_forward(net, x)
        s = (pre > 0).astype(np.uint8)
        A, aF = arch.res_compose(net, s)
        xt = np.append(x, 1.0)
        np.testing.assert_allclose(A @ xt, pre, atol=1e-12)
        assert abs(aF @ xt - F) < 1e-12
        X = torch.tensor(x[None, :], requires_grad=True)
        _, Ft = _torch_F(net, X)
        Ft.sum().backward()
        np.testing.assert_allclose(aF[:3], X.grad[0].numpy(), atol=1e-12)


def _brute_faces(arch, pool, box):
    """{key: interior point} of every non-empty face, by LP over every (pattern, index)."""
    out = {}
    N, M = pool.N, pool.M
    for code in range(1 << N):
        s = np.array([(code >> k) & 1 for k in range(N)], dtype=np.uint8)
        rows, aFs, off = [], [], 0
        for n in pool.subnets:
            A, aF = _frozen_maps(n, s[off:off + n.N])
            rows.append(A * (1.0 - 2.0 * s[off:off + n.N])[:, None])
            aFs.append(aF)
            off += n.N
        for j in range(M):
            if np.linalg.norm(aFs[j][:3]) == 0:
                continue
            C = np.vstack(rows + [(aFs[i] - aFs[j])[None, :] for i in range(M) if i != j])
            zero = np.linalg.norm(C[:, :3], axis=1) == 0
            if np.any(C[zero, 3] > 0):
                continue
            t, x = pins.chebyshev_lp(C[~zero], box, plane=aFs[j])
            if t > 1e-9:
                out[code | (j << N)] = x
    return out


def _check_polygons(arch, pool, mesh, box):
    for f in mesh.faces:
        s, j = pool.split(f.key)
        C, ids, aF = pool.cell_rows(s, j, box)
        V3 = pins.halfspace_polygon(C, aF, f.verts.mean(0), box)
        assert len(V3) == len(f.verts)
        for v in f.verts:
            assert np.min(np.linalg.norm(V3 - v, axis=1)) < 1e-8


def _check_reciprocal_edges(arch, pool, mesh):
    """Every inner edge of a face is an edge of the cell across it, reversed (closed surface)."""
    by_key = mesh.by_key()
    for f in mesh.faces:
        m = len(f.edges)
        for i, e in enumerate(f.edges):
            nk = pool.neighbour(f.key, e)
            if nk is None:
                continue
            g = by_key.get(nk)
            assert g is not None, "the cell across an edge has no face"
            back = e if e < pool.N else pool.N + (f.key >> pool.N)
            a, b = f.verts[i], f.verts[(i + 1) % m]
            ok = False
            for k, e2 in enumerate(g.edges):
                c, d = g.verts[k], g.verts[(k + 1) % len(g.edges)]
                if e2 == back and np.linalg.norm(c - b) < 1e-9 and np.linalg.norm(d - a) < 1e-9:
                    ok = True
            assert ok, "edge without its reversed twin"


@pytest.mark.parametrize("make", [
    lambda A: A.MaxPool([_resnet(A, 11, first=3, mid=3, with_id=True, depth=2),
                         _resnet(A, 12, first=2, mid=2, with_id=False, with_v=True, depth=2)]),
    lambda A: A.as_pool(_resnet(A, 13, first=3, mid=3)),
])
def test_march_finds_every_face_of_a_tiny_network(arch, make):
    pool = make(arch)
    assert pool.N <= 10
    box = 1.5
    brute = _brute_faces(arch, pool, box)
    assert brute
    mesh = arch.march(pool, list(brute.items()), box)
    assert not mesh.failed
    assert {f.key for f in mesh.faces} == set(brute)
    _check_polygons(arch, pool, mesh, box)


def test_pooled_polytopes_are_their_intersection(arch):
    # max of two max-of-planes nets is the max over all 24 planes: the intersection polytope
    p1, p2 = polytope_max_of_planes(seed=1), polytope_max_of_planes(seed=2)
    pool = arch.MaxPool([_from_mlp(arch, p1), _from_mlp(arch, p2)])
    normals = np.vstack([p1.meta["normals"], p2.meta["normals"]])
    area, vol, verts = pins.polytope_facets(normals, 0.5)
    seed = arch.seed_ray(pool, np.zeros(3), np.array([1.0, 0.37, 0.21]) / np.linalg.norm([1.0, 0.37, 0.21]))
    assert seed is not None
    mesh = arch.march(pool, [seed])
    assert not mesh.failed and mesh.degenerate == 0
    assert abs(sum(f.area() for f in mesh.faces) - area.sum()) < 1e-9
    # divergence theorem per face: V = 1/3 sum area_f (n_f . p_f), n_f the outward unit normal
    v = sum(f.area() * (f.aF[:3] / np.linalg.norm(f.aF[:3])) @ f.verts[0] for f in mesh.faces) / 3.0
    assert abs(v - vol) < 1e-9
    for p in verts:                                 # every polytope corner is a mesh vertex
        assert min(np.min(np.linalg.norm(f.verts - p, axis=1)) for f in mesh.faces) < 1e-9
    _check_reciprocal_edges(arch, pool, mesh)
    # both sub-networks carry faces, and some edges are pooling rows
    assert {f.key >> pool.N for f in mesh.faces} == {0, 1}
    assert any(e >= pool.N and e < pool.N + pool.M for f in mesh.faces for e in f.edges)


def test_residual_surface_is_closed(arch):
    net = _resnet(arch, 21, first=6, mid=6)
    pool = arch.as_pool(net)
    seed = arch.seed_ray(pool, np.zeros(3), np.array([1.0, 0.0, 0.0]))
    assert seed is not None
    mesh = arch.march(pool, [seed])
    assert mesh.faces and not mesh.failed
    assert all(e < pool.N for f in mesh.faces for e in f.edges), "the surface leaves the box"
    _check_reciprocal_edges(arch, pool, mesh)
    for f in mesh.faces:                            # F vanishes on every face, by torch
        _, F = _torch_F(net, f.verts)
        assert np.abs(F.detach().numpy()).max() < 1e-12


def test_planted_mistakes_are_caught(arch, monkeypatch):
    # dropping the shortcut from the compose, or flipping the pooling rows, fails a pin
    net = _resnet(arch, 3)
    s = np.random.default_rng(0).integers(0, 2, net.N).astype(np.uint8)
    orig = arch.res_compose

    def no_shortcut(n, st):
        return orig(arch.ResNet(n.weights, n.biases, n.w_out, n.b_out, {}), st)
    monkeypatch.setattr(arch, "res_compose", no_shortcut)
    assert not np.allclose(arch.res_compose(net, s)[0], _frozen_maps(net, s)[0], atol=1e-12)
    monkeypatch.setattr(arch, "res_compose", orig)

    p1, p2 = polytope_max_of_planes(seed=1), polytope_max_of_planes(seed=2)
    pool = arch.MaxPool([_from_mlp(arch, p1), _from_mlp(arch, p2)])
    rows = arch.MaxPool.cell_rows

    def flipped(self, s, j, box=1.5):
        C, ids, aF = rows(self, s, j, box)
        for r, i in enumerate(ids):
            if self.N <= i < self.N + self.M:
                C[r] = -C[r]
        return C, ids, aF
    monkeypatch.setattr(arch.MaxPool, "cell_rows", flipped)
    area, _, _ = pins.polytope_facets(np.vstack([p1.meta["normals"], p2.meta["normals"]]), 0.5)
    seed = arch.seed_ray(pool, np.zeros(3), np.array([1.0, 0.37, 0.21]) / np.linalg.norm([1.0, 0.37, 0.21]))
    mesh = arch.march(pool, [seed])
    assert mesh.failed or abs(sum(f.area() for f in mesh.faces) - area.sum()) > 1e-6


@pytest.mark.parametrize("slope", [0.1, 0.3])
def test_leaky_relu(arch, slope):
    # forward and gradient by torch's leaky_relu, cell maps by the frozen network, every face
    # of a tiny net by LP, and a closed surface on a larger one
    import torch
    net = _resnet(arch, 31, first=3, mid=3)
    net.slope = slope
    net.b_out = 0.0
    net.b_out = -0.5 - arch.res_forward(net, np.zeros(3))[1]
    rng = np.random.default_rng(32)
    for x in rng.uniform(-1.0, 1.0, size=(15, 3)):
        pre, F = arch.res_forward(net, x)
        p_t, F_t = _torch_F(net, x)
        np.testing.assert_allclose(pre, p_t.detach().numpy()[0], atol=1e-13)
        assert abs(F - float(F_t.detach()[0])) < 1e-13
        s = (pre > 0).astype(np.uint8)
        A, aF = arch.res_compose(net, s)
        A2, aF2 = _frozen_maps(net, s)
        np.testing.assert_allclose(A, A2, atol=1e-12)
        np.testing.assert_allclose(aF, aF2, atol=1e-12)
        assert abs(aF @ np.append(x, 1.0) - F) < 1e-12
        X = torch.tensor(x[None, :], requires_grad=True)
        _torch_F(net, X)[1].sum().backward()
        np.testing.assert_allclose(aF[:3], X.grad[0].numpy(), atol=1e-12)
    pool = arch.as_pool(net)
    brute = _brute_faces(arch, pool, 1.5)
    mesh = arch.march(pool, list(brute.items()))
    assert brute and not mesh.failed and {f.key for f in mesh.faces} == set(brute)
    _check_polygons(arch, pool, mesh, 1.5)
    big = _resnet(arch, 21, first=6, mid=6)
    big.slope = slope
    big.b_out = 0.0
    big.b_out = -0.5 - arch.res_forward(big, np.zeros(3))[1]
    bp = arch.as_pool(big)
    m = arch.march(bp, [arch.seed_ray(bp, np.zeros(3), np.array([1.0, 0.0, 0.0]))])
    assert m.faces and not m.failed
    if all(e < bp.N for f in m.faces for e in f.edges):
        _check_reciprocal_edges(arch, bp, m)


def test_leaky_slope_is_caught_when_dropped(arch, monkeypatch):
    # a compose that ignores the slope (plain ReLU masks) fails the frozen-network pin
    net = _resnet(arch, 33, first=3, mid=3)
    net.slope = 0.2
    s = np.random.default_rng(1).integers(0, 2, net.N).astype(np.uint8)
    orig = arch.res_compose

    def plain(n, st):
        return orig(arch.ResNet(n.weights, n.biases, n.w_out, n.b_out, n.shortcuts, 0.0), st)
    monkeypatch.setattr(arch, "res_compose", plain)
    assert not np.allclose(arch.res_compose(net, s)[1], _frozen_maps(net, s)[1], atol=1e-12)
