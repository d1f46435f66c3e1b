"""Pins for the oracle of the learned constraint proposal (CPU only).

The gradients are pinned by central finite differences of the loss, the loss by its closed
form at a constant network, and the training features by the geometry of exact faces (the
entry point lies on the face plane, the labels are the face's edge neurons)."""
import numpy as np
import pytest

from oracle import proposal as P
from synth import polytope_max_of_planes, tiny_net


def _data(rng, B, n_in, n_out):
    X = rng.normal(size=(B, n_in))
    Y = (rng.uniform(size=(B, n_out)) < 0.2).astype(np.float64)
    return X, Y


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    prm = P.init_params(9, 16, 12, seed=1)
    for k in prm:                       # non-zero biases so that every term is exercised
        prm[k] = prm[k] + 0.1 * rng.normal(size=prm[k].shape)
    X, Y = _data(rng, 8, 9, 12)
    z, cache = P.forward(prm, X)
    g = P.backward(prm, z, Y, cache)
    h = 1e-6
    for name, W in prm.items():
        flat = W.reshape(-1)
        for i in rng.choice(flat.size, min(flat.size, 25), replace=False):
            old = flat[i]
            flat[i] = old + h
            lp = P.loss(P.forward(prm, X)[0], Y)
            flat[i] = old - h
            lm = P.loss(P.forward(prm, X)[0], Y)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name].reshape(-1)[i]) <= 1e-7 + 1e-5 * abs(fd), (name, i)


def test_loss_and_bias_gradient_closed_form_at_constant_net():
    # with every weight zero the logits are b3 for every sample: the loss is
    # mean_k softplus(b3_k) - mean(Y) b3 and dL/db3_k = (sigmoid(b3_k) - mean_b Y_bk) / n_out
    rng = np.random.default_rng(2)
    prm = P.init_params(5, 7, 6, seed=3)
    for k in ("W1", "W2", "W3"):
        prm[k][:] = 0.0
    prm["b3"] = rng.normal(size=6)
    X, Y = _data(rng, 10, 5, 6)
    z, cache = P.forward(prm, X)
    b3 = prm["b3"]
    want = np.mean(np.log1p(np.exp(b3))) - np.mean(Y * b3[None, :])
    assert abs(P.loss(z, Y) - want) < 1e-14
    g = P.backward(prm, z, Y, cache)
    np.testing.assert_allclose(g["b3"], (1 / (1 + np.exp(-b3)) - Y.mean(0)) / 6, rtol=1e-13)
    assert not np.any(g["W1"]) and not np.any(g["W2"])


def test_initial_scores_match_sparse_labels():
    prm = P.init_params(11, 32, 40, seed=0)
    assert np.allclose(1 / (1 + np.exp(-prm["b3"])), 1 / 32)


@pytest.mark.parametrize("make,ray", [(polytope_max_of_planes, [1.0, 0.0, 0.0]),
                                      (lambda: tiny_net((8, 8), 11), [1.0, 0.37, 0.21])])
def test_face_samples_geometry(oracle_mod, make, ray):
    mlp = make()
    d = np.asarray([ray]) / np.linalg.norm(ray)
    net, mesh = oracle_mod.mesh_from_rays(mlp, np.zeros((1, 3)), d)
    X, Y, tags = P.face_samples(mesh, mlp.widths)
    assert len(X) == sum(len(f.edges) for f in mesh.faces) > 0
    by_key = mesh.by_key()
    for x, y, (key, e) in zip(X, Y, tags):
        f = by_key[key]
        n, off = x[3:6], x[6]
        assert abs(np.linalg.norm(n) - 1.0) < 1e-12
        assert abs(n @ x[:3] + off) < 1e-9                 # the entry point lies on the face plane
        assert np.all(f.verts @ n + off > -1e-9) and np.all(f.verts @ n + off < 1e-9)
        g = f.aF[:3]                                      # oriented like grad F
        assert n @ g > 0
        assert set(np.flatnonzero(y)) == {p for p in f.edges if p < mlp.N}
        r = 0
        for l, w in enumerate(mlp.widths):               # per-layer active fractions of the key
            assert x[7 + l] == bin((key >> r) & ((1 << w) - 1)).count("1") / w
            r += w
        # the entry point is the midpoint of the edge carried by plane e
        j = f.edges.index(e)
        np.testing.assert_allclose(x[:3], 0.5 * (f.verts[j] + f.verts[(j + 1) % len(f.edges)]), atol=1e-15)
