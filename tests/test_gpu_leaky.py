"""Leaky / parametric ReLU nets on the device (the activation the paper's closing remarks name
next): g(a) = a for a > 0, slope * a otherwise.  The cells are Def. 2's; inside a cell the masks
diag(s_l) of Cor. 1 become diag(s_l + slope (1 - s_l)), and the triggers' forward pass and
gradient take the slope.  The GPU mesh must be the oracle's (oracle/arch.py, the same net as a
residual-free ResNet with that slope) face for face.  Needs a GPU."""
import numpy as np
import pytest

from oracle import arch
from synth import leaky, sphere_net, tiny_net
from tests import parity

pytestmark = pytest.mark.gpu
X_RAY = np.array([[1.0, 0.0, 0.0]])
ORIGIN = np.zeros((1, 3))


def _oracle_mesh(oracle_mod, mlp):
    net = arch.ResNet(weights=mlp.weights, biases=mlp.biases, w_out=mlp.w_out, b_out=mlp.b_out, slope=mlp.slope)
    pool = arch.as_pool(net)
    ref = arch.march(pool, [arch.seed_ray(pool, ORIGIN[0], X_RAY[0])])
    # the pooled oracle numbers the box planes after its M = 1 pooling row: N + 1 + k -> N + k
    for f in ref.faces:
        f.edges = [e - 1 if e > mlp.N else e for e in f.edges]
    return ref


@pytest.mark.parametrize("make", [lambda: leaky(sphere_net(seed=21, width=32, depth=4), 0.1),
                                  lambda: leaky(sphere_net(seed=21, width=32, depth=4), 0.25),
                                  lambda: leaky(tiny_net((8, 8), 11), 0.2)])
@pytest.mark.parametrize("precision,schedule", [("fp64", "persistent"), ("fp64", "levels"), ("mixed", "persistent")])
def test_leaky_mesh_matches_oracle(oracle_mod, make, precision, schedule):
    import paper_2106_10031_gb300 as am
    mlp = make()
    ref = _oracle_mesh(oracle_mod, mlp)
    with am.Mesher(max_cells=1 << 17, max_neurons=max(64, mlp.N), max_width=max(mlp.widths)) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, ORIGIN, X_RAY)
        m.march(precision=precision, schedule=schedule)
        mesh = m.get_mesh(nid)
        st = m.stats()
    r = parity.compare(ref, mesh, mlp.N, rtol=1e-9)
    print(f"\n{mlp.name} {precision}/{schedule}: {r['faces']} faces, max rel vertex err {r['max_rel_vertex_err']:.2e}")
    assert st["degenerate"] == 0 and r["faces"] == len(ref.faces)
    if precision == "mixed":
        assert st["refined_cells"] == st["cells"]          # leaky nets march in FP64


def test_leaky_refusals_and_triggers(oracle_mod):
    import paper_2106_10031_gb300 as am
    mlp = leaky(sphere_net(seed=21, width=32, depth=4), 0.1)
    with am.Mesher(max_cells=1 << 17, max_neurons=256, max_width=32) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, ORIGIN, X_RAY)
        with pytest.raises(am.AMError):
            m.march(precision="sliced")                     # the sliced operands mask with s_l alone
        keys = np.zeros((1, (mlp.N + 63) // 64), dtype=np.uint64)
        with pytest.raises(am.AMError):
            m.compose(nid, keys, "mixed")
        rows, _ = m.compose(nid, keys, "fp64")
        # sphere tracing uses the leaky gradient: its seeds lie on the surface, in the oracle's cells
        starts = np.array([[1.2, 0.1, -0.2], [-0.3, 1.1, 0.4], [0.2, -0.4, -1.2]])
        m.reset()
        _, pts = m.seed_sphere_trace(nid, starts, eta=1.0, max_steps=64, eps=1e-12)
    net = arch.ResNet(weights=mlp.weights, biases=mlp.biases, w_out=mlp.w_out, b_out=mlp.b_out, slope=mlp.slope)
    # the all-inactive pattern: every layer passes slope * its pre-activation
    A, aF = arch.res_compose(net, np.zeros(mlp.N, dtype=np.uint8))
    ref = np.vstack([A, aF[None, :]])
    assert np.abs(rows[0] - ref).max() <= 1e-12 * (1.0 + np.abs(ref).max())
    ok = ~np.isnan(pts[:, 0])
    assert ok.any()
    for p in pts[ok]:
        _, F = arch.res_forward(net, p)
        assert abs(F) < 1e-9
