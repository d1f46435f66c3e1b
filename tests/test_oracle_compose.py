"""Pins for the oracle's forward pass (Eq. 1), state functional (Def. 2) and region-wise
affine maps (Lemma 1, Cor. 1).  CPU only."""
import numpy as np
import pytest

from synth import decoder_net, octahedron, polytope_max_of_planes, sphere_net, tiny_net
from tests import pins

NETS = [
    lambda: octahedron(),
    lambda: polytope_max_of_planes(),
    lambda: tiny_net((8, 8), seed=11),
    lambda: sphere_net(),
    lambda: decoder_net(width=24, depth=6, latent_dim=9, skip_layer=3, seed=7),
]


@pytest.mark.parametrize("make", NETS)
def test_forward_matches_torch(oracle_mod, make):
    mlp = make()
    net = oracle_mod.OracleNet(mlp)
    X = np.random.default_rng(0).uniform(-1.5, 1.5, (20, 3))
    pre_t, F_t = pins.torch_forward(mlp, X)
    for x, p, f in zip(X, pre_t, F_t):
        pre, F = net.forward(x)
        np.testing.assert_allclose(pre, p, rtol=1e-12, atol=1e-12)
        assert abs(F - f) <= 1e-12 * (1 + abs(f))


def test_state_tie_is_zero(oracle_mod):
    # Def. 2: a_lk(x) = 0 gives s_lk = 0.  At the origin the octahedron's relu(x_i) neurons tie.
    net = oracle_mod.OracleNet(octahedron())
    assert net.state(np.zeros(3)).tolist() == [0, 0, 0, 1, 1, 1]
    pre, F = net.forward(np.zeros(3))
    assert pre[:3].tolist() == [0.0, 0.0, 0.0] and F == -1.0


@pytest.mark.parametrize("make", NETS)
def test_compose_equals_masked_network(oracle_mod, make):
    # Lemma 1 / Cor. 1: for ANY pattern s the composed rows are the affine maps of the
    # network with its states frozen to s (evaluated here at 0, e_x, e_y, e_z).
    mlp = make()
    net = oracle_mod.OracleNet(mlp)
    rng = np.random.default_rng(1)
    for _ in range(10):
        s = rng.integers(0, 2, mlp.N).astype(np.uint8)
        A, aF = net.compose(s)
        A_ref, aF_ref = pins.masked_affine_maps(mlp, s)
        scale = 1 + np.abs(A_ref).max()
        np.testing.assert_allclose(A, A_ref, rtol=0, atol=1e-11 * scale)
        np.testing.assert_allclose(aF, aF_ref, rtol=0, atol=1e-11 * (1 + np.abs(aF_ref).max()))


def test_layer1_rows_closed_form(oracle_mod):
    # Cor. 1 for l = 1: a_1k = pi_k W_1 (plus the latent's constant and the bias).
    mlp = decoder_net(width=16, depth=4, latent_dim=5, skip_layer=2, seed=3)
    net = oracle_mod.OracleNet(mlp)
    s = np.random.default_rng(2).integers(0, 2, mlp.N).astype(np.uint8)
    A, _ = net.compose(s)
    W1, b1 = mlp.weights[0], mlp.biases[0]
    np.testing.assert_allclose(A[:16, :3], W1[:, :3], rtol=0, atol=0)
    np.testing.assert_allclose(A[:16, 3], b1 + W1[:, 3:] @ mlp.latent, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("make", NETS)
def test_compose_reproduces_F_and_gradient_in_own_cell(oracle_mod, make):
    # At a point x of region r: A^r [x;1] = a(x), a_F^r [x;1] = F(x), a_F^r[0:3] = grad F(x)
    # (central differences inside the cell), and sign(A^r [x;1]) reproduces s(x).
    mlp = make()
    net = oracle_mod.OracleNet(mlp)
    rng = np.random.default_rng(3)
    tested = 0
    for x in rng.uniform(-1.2, 1.2, (60, 3)):
        pre, F = net.forward(x)
        margin = np.min(np.abs(pre))
        if margin < 1e-4:
            continue
        s = (pre > 0).astype(np.uint8)
        A, aF = net.compose(s)
        xt = np.append(x, 1.0)
        np.testing.assert_allclose(A @ xt, pre, rtol=1e-10, atol=1e-10)
        assert abs(aF @ xt - F) < 1e-10 * (1 + abs(F))
        # a step that cannot leave the cell: every pre-activation moves by less than margin/4
        h = 0.25 * margin / max(1.0, float(np.linalg.norm(A[:, :3], axis=1).max()))
        g = np.array([(net.F(x + h * e) - net.F(x - h * e)) / (2 * h) for e in np.eye(3)])
        np.testing.assert_allclose(aF[:3], g, rtol=1e-6, atol=1e-12 * (1 + abs(F)) / h)   # round-off only
        assert np.array_equal((A @ xt > 0).astype(np.uint8), s)
        tested += 1
    assert tested >= 10
