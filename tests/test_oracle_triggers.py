"""Pins of the oracle's customised triggers (Sec. 4.3): the sphere-tracing walk for an SDF
(Sec. 4.3.1) and the random-pair dichotomy (Sec. 4.3.2).  CPU only.

Independent routes: the max-of-planes polytope gives closed forms (one step with eta = 1
from 1.5 n_i is the orthogonal projection 0.5 n_i onto facet i; the segment from the centre to
1.5 n_i crosses the surface at 0.5 n_i); torch FP64 autograd gives F and its gradient for the
update rule; the pairing rule is checked on a hand-made sign list."""
import numpy as np
import pytest

from synth import polytope_max_of_planes, sphere_net, tiny_net, trigger_points
from tests import pins


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod


def _torch_F_grad(mlp, x):
    """F and grad F at x by torch autograd (FP64), independent of the oracle."""
    import torch
    import torch.nn.functional as tf
    X = torch.tensor(np.asarray(x, dtype=np.float64)[None, :], requires_grad=True)
    h = X
    for l, (W, b) in enumerate(zip(mlp.weights, mlp.biases), start=1):
        inp = h if l != mlp.skip_layer else torch.cat([h, X], 1)
        h = torch.relu(tf.linear(inp, torch.as_tensor(W), torch.as_tensor(b)))
    F = (h[0] * torch.as_tensor(mlp.w_out)).sum() + mlp.b_out
    F.backward()
    return float(F.detach()), X.grad[0].numpy().copy()


@pytest.mark.parametrize("eta,land", [(1.0, 0.5), (0.5, 1.0), (0.25, 1.25)])
def test_step_on_the_polytope_is_the_closed_form(orc, eta, land):
    # F = n_i . x - 1/2 near 1.5 n_i with |grad F| = 1: one step moves by eta * F along -n_i
    mlp = polytope_max_of_planes()
    net = orc.OracleNet(mlp)
    for n in mlp.meta["normals"]:
        rc, x, F, g, t = net.sphere_trace(1.5 * n, eta, 1, 0.0)
        assert rc == 0 and t == 1
        np.testing.assert_allclose(x, land * n, atol=1e-12)
        np.testing.assert_allclose(g, n, atol=1e-12)
        assert abs(F - (land - 0.5)) < 1e-12


def test_step_is_the_update_rule_with_the_autograd_gradient(orc):
    # x_1 = x_0 - eta F(x_0) grad F(x_0), F and grad F from torch autograd
    mlp = sphere_net(seed=21, width=32, depth=4, sigma=0.05)
    net = orc.OracleNet(mlp)
    for x0 in trigger_points(12, seed=3, box=1.2):
        F0, g0 = _torch_F_grad(mlp, x0)
        for eta in (1.0, 0.7):
            rc, x1, F1, g1, t = net.sphere_trace(x0, eta, 1, 0.0)
            assert rc == 0 and t == 1
            np.testing.assert_allclose(x1, x0 - eta * F0 * g0, rtol=0, atol=1e-12)
            Fx, gx = _torch_F_grad(mlp, x1)
            assert abs(F1 - Fx) < 1e-12
            np.testing.assert_allclose(g1, gx, atol=1e-12)


def test_walk_stops_at_eps_or_the_step_budget(orc):
    mlp = sphere_net(seed=21, width=32, depth=4, sigma=0.05)
    net = orc.OracleNet(mlp)
    rc, x, F, g, t = net.sphere_trace([1.2, 0.3, 0.1], 1.0, 200, 1e-12)
    assert rc == 0 and abs(F) <= 1e-12 and 0 < t < 200
    assert abs(pins.torch_forward(mlp, x)[1][0]) <= 1e-12
    rc, x2, F2, g2, t2 = net.sphere_trace([1.2, 0.3, 0.1], 1.0, 3, 1e-12)
    assert rc == 0 and t2 == 3 and abs(F2) > 1e-12
    rc, x3, F3, g3, t3 = net.sphere_trace([1.2, 0.3, 0.1], 1.0, 0, 1e-12)
    assert t3 == 0 and np.array_equal(x3, [1.2, 0.3, 0.1])


def test_flat_cell_is_reported(orc):
    # every hidden unit dead everywhere (W_1 = 0, b_1 = -1): F is constant, grad F = 0, and
    # the walk cannot move
    mlp = tiny_net((4, 4), 3)
    mlp.weights[0][:] = 0.0
    mlp.biases[0][:] = -1.0
    net = orc.OracleNet(mlp)
    rc, x, F, g, t = net.sphere_trace([0.3, 0.2, 0.1], 1.0, 10, 0.0)
    assert rc == -6 and t == 0


def test_traced_seed_lies_on_the_surface_in_its_cell(orc):
    mlp = sphere_net(seed=21, width=32, depth=4, sigma=0.05)
    net = orc.OracleNet(mlp)
    starts = trigger_points(16, seed=4, box=1.4)
    seeds = orc.seed_sphere_trace(net, starts, eta=1.0, max_steps=200, eps=1e-12)
    found = [s for s in seeds if s is not None]
    assert len(found) >= 14
    for key, xs in found:
        pre, F = pins.torch_forward(mlp, xs)
        assert abs(F[0]) <= 1e-12
        # the seed point is the exact root inside the seed cell: its pattern is the key
        # (up to rows tight at the point, which the strict sign can put on either side)
        s = orc.key_to_state(key, mlp.N)
        ok = (pre[0] > 0) == (s == 1)
        assert np.all(ok | (np.abs(pre[0]) < 1e-12))


def test_sign_pairs_rule(orc):
    F = [1.0, -1.0, 0.0, -2.0, 3.0, 4.0, -0.5]
    assert orc.sign_pairs(F, 10) == [(1, 0), (3, 4), (6, 5)]
    assert orc.sign_pairs(F, 1) == [(1, 0)]
    assert orc.sign_pairs([0.0, 1.0, 2.0], 5) == []


def test_pair_dichotomy_on_the_polytope_is_the_closed_form(orc):
    # F(0) = -1/2 and F(1.5 n_i) = 1: the crossing on that segment is the facet's foot 0.5 n_i
    mlp = polytope_max_of_planes()
    net = orc.OracleNet(mlp)
    N = mlp.meta["normals"]
    pts = []
    for n in N[:6]:
        pts += [1.5 * n, np.zeros(3)]
    seeds = orc.seed_pairs(net, np.array(pts), 100)
    assert len(seeds) == 6
    for (key, xs), n in zip(seeds, N[:6]):
        np.testing.assert_allclose(xs, 0.5 * n, atol=1e-12)


def test_random_pairs_reach_every_component(orc):
    # a net whose zero set has two components: random pairs seed both, and the march from all
    # the seeds is the union of the marches from each seed alone
    mlp = tiny_net((8, 8), 1, sigma=0.3)
    net = orc.OracleNet(mlp)
    pts = trigger_points(300, seed=7, box=1.5)
    seeds = [s for s in orc.seed_pairs(net, pts, 48) if s is not None]
    assert len(seeds) >= 32
    for key, xs in seeds:
        assert abs(pins.torch_forward(mlp, xs)[1][0]) <= 1e-12
    comps = []
    for sd in seeds:
        if not any(sd[0] in c for c in comps):
            comps.append({f.key for f in orc.march(net, [sd]).faces})
    assert len(comps) >= 2
    whole = orc.march(net, seeds)
    assert {f.key for f in whole.faces} == set().union(*comps) and not whole.failed
