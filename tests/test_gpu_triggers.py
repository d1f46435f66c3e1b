"""The customised triggers on the device (Sec. 4.3) against the oracle: sphere tracing for an
SDF (Sec. 4.3.1) and the random-pair dichotomy (Sec. 4.3.2).  Needs a GPU."""
import numpy as np
import pytest

from synth import polytope_max_of_planes, sphere_net, tiny_net, trigger_points
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def am():
    import paper_2106_10031_gb300 as am_mod
    return am_mod


def _ref_points(seeds, n):
    out = np.full((n, 3), np.nan)
    for i, s in enumerate(seeds):
        if s is not None:
            out[i] = s[1]
    return out


def _check_points(got, ref):
    assert np.array_equal(np.isnan(got[:, 0]), np.isnan(ref[:, 0]))
    ok = ~np.isnan(ref[:, 0])
    np.testing.assert_allclose(got[ok], ref[ok], rtol=0, atol=1e-9)


@pytest.mark.parametrize("make,eta", [
    (polytope_max_of_planes, 1.0),
    (lambda: sphere_net(seed=21, width=32, depth=4, sigma=0.05), 1.0),
    (lambda: sphere_net(seed=21, width=32, depth=4, sigma=0.05), 0.6),
])
def test_sphere_trace_matches_oracle(oracle_mod, am, make, eta):
    mlp = make()
    net = oracle_mod.OracleNet(mlp)
    starts = trigger_points(40, seed=4, box=1.4)
    seeds = oracle_mod.seed_sphere_trace(net, starts, eta=eta, max_steps=200, eps=1e-12)
    live = [s for s in seeds if s is not None]
    assert len(live) >= 30
    ref = oracle_mod.march(net, live)
    with am.Mesher(max_cells=1 << 17, max_neurons=256, max_width=64) as m:
        nid = m.load_mlp(mlp)
        n_new, pts = m.seed_sphere_trace(nid, starts, eta=eta, max_steps=200, eps=1e-12)
        assert n_new == len({k for k, _ in live})
        _check_points(pts, _ref_points(seeds, len(starts)))
        m.march()
        parity.compare(ref, m.get_mesh(nid), mlp.N, rtol=1e-9)


def test_random_pairs_reach_both_components(oracle_mod, am):
    # a net whose zero set has two components; the pairs seed both, and the mesh of the march
    # from them is the oracle's
    mlp = tiny_net((8, 8), 1, sigma=0.3)
    net = oracle_mod.OracleNet(mlp)
    pts = trigger_points(300, seed=7, box=1.5)
    seeds = oracle_mod.seed_pairs(net, pts, 48)
    live = [s for s in seeds if s is not None]
    ref = oracle_mod.march(net, live)
    with am.Mesher(max_cells=1 << 16, max_neurons=64, max_width=64) as m:
        nid = m.load_mlp(mlp)
        n_pairs, n_new, got = m.seed_pairs(nid, pts, 48)
        assert n_pairs == len(seeds) == 48
        assert n_new == len({k for k, _ in live})
        _check_points(got, _ref_points(seeds, n_pairs))
        m.march()
        parity.compare(ref, m.get_mesh(nid), mlp.N, rtol=1e-9)


@pytest.mark.parametrize("n_points,max_pairs", [(3001, 5000), (2500, 700), (7, 3)])
def test_pairing_across_chunks(oracle_mod, am, n_points, max_pairs):
    # the pairing is exact index work: the segments, hence the seed points, are the oracle's,
    # with the samples spanning several 1024-sample chunks and a ragged tail
    mlp = polytope_max_of_planes()
    net = oracle_mod.OracleNet(mlp)
    pts = trigger_points(n_points, seed=11, box=1.2)
    seeds = oracle_mod.seed_pairs(net, pts, max_pairs)
    with am.Mesher(max_cells=1 << 16, max_neurons=64, max_width=64) as m:
        nid = m.load_mlp(mlp)
        n_pairs, n_new, got = m.seed_pairs(nid, pts, max_pairs)
        assert n_pairs == len(seeds)
        _check_points(got, _ref_points(seeds, n_pairs))


def test_trigger_edge_cases(am):
    mlp = polytope_max_of_planes()
    with am.Mesher(max_cells=1 << 12, max_neurons=64, max_width=64) as m:
        nid = m.load_mlp(mlp)
        # every sample outside the polytope: no pair
        far = np.array([[1.4, 1.4, 1.4], [-1.4, 1.4, 1.4], [1.4, -1.4, -1.4]])
        with pytest.raises(am.AMError) as e:
            m.seed_pairs(nid, far, 4)
        assert e.value.status == 5
        for bad in (dict(eta=0.0), dict(eta=1.5), dict(max_steps=-1), dict(eps=-1.0)):
            with pytest.raises(am.AMError) as e:
                m.seed_sphere_trace(nid, far, **bad)
            assert e.value.status == 1
        # a start already on a facet's foot: F = 0 there, no step, the padded segment finds it
        n0 = mlp.meta["normals"][0]
        n_new, p = m.seed_sphere_trace(nid, [0.5 * n0], max_steps=0)
        assert n_new == 1 and np.abs(p[0] - 0.5 * n0).max() < 1e-9
    flat = tiny_net((4, 4), 3)
    flat.weights[0][:] = 0.0
    flat.biases[0][:] = -1.0
    with am.Mesher(max_cells=1 << 12, max_neurons=64, max_width=64) as m:
        nid = m.load_mlp(flat)
        with pytest.raises(am.AMError) as e:
            m.seed_sphere_trace(nid, [[0.3, 0.2, 0.1]])
        assert e.value.status == 5
