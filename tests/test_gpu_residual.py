"""Residual blocks on the device (Sec. 5.1): hidden layer q adds S_q h_src to its pre-activation,
the identity from an earlier hidden layer (first kind, g(x + T x)) or a matrix V from the input
(second kind, g(V x + T x)).  Inside a cell the compose gains the masked term S_q diag(g) Z_src
(the region-wise map of a residual block), and the triggers' forward pass and gradient carry
the shortcut.  The GPU mesh must be the oracle's (oracle/arch.py, the same net as a ResNet)
face for face, in both schedules and with the mixed precision falling back to FP64.  Needs a
GPU."""
import numpy as np
import pytest

from oracle import arch
from synth import leaky, residual_net
from tests import parity

pytestmark = pytest.mark.gpu
X_RAY = np.array([[1.0, 0.0, 0.0]])
ORIGIN = np.zeros((1, 3))


def _resnet(mlp):
    return arch.ResNet(weights=mlp.weights, biases=mlp.biases, w_out=mlp.w_out, b_out=mlp.b_out,
                       shortcuts=dict(mlp.shortcuts), slope=mlp.slope)


def _oracle_mesh(mlp):
    pool = arch.as_pool(_resnet(mlp))
    ref = arch.march(pool, [arch.seed_ray(pool, ORIGIN[0], X_RAY[0])])
    assert ref.faces and not ref.failed
    # the pooled oracle numbers the box planes after its M = 1 pooling row: N + 1 + k -> N + k
    for f in ref.faces:
        f.edges = [e - 1 if e > mlp.N else e for e in f.edges]
    return ref


NETS = [lambda: residual_net(seed=40, width=12, depth=6),
        lambda: residual_net(seed=32, width=24, depth=6),
        lambda: leaky(residual_net(seed=32, width=24, depth=6), 0.1)]


@pytest.mark.parametrize("make", NETS)
@pytest.mark.parametrize("precision,schedule", [("fp64", "persistent"), ("fp64", "levels"), ("mixed", "persistent")])
def test_residual_mesh_matches_oracle(oracle_mod, make, precision, schedule):
    import paper_2106_10031_gb300 as am
    mlp = make()
    ref = _oracle_mesh(mlp)
    with am.Mesher(max_cells=1 << 17, max_neurons=max(64, mlp.N), max_width=max(mlp.widths)) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, ORIGIN, X_RAY)
        m.march(precision=precision, schedule=schedule)
        mesh = m.get_mesh(nid)
        st = m.stats()
    r = parity.compare(ref, mesh, mlp.N, rtol=1e-9)
    print(f"\n{mlp.name} {precision}/{schedule}: {r['faces']} faces, max rel vertex err {r['max_rel_vertex_err']:.2e}")
    assert st["degenerate"] == 0 and r["faces"] == len(ref.faces)
    if mlp.slope == 0.0:
        assert mesh.n_open_faces == 0                      # (the leaky variant's surface leaves the box)
    if precision == "mixed":
        assert st["refined_cells"] == st["cells"]          # nets with hidden shortcuts march in FP64


def test_residual_compose_refusals_and_triggers(oracle_mod):
    import paper_2106_10031_gb300 as am
    mlp = residual_net(seed=32, width=24, depth=6)
    net = _resnet(mlp)
    rng = np.random.default_rng(5)
    with am.Mesher(max_cells=1 << 17, max_neurons=256, max_width=32) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, ORIGIN, X_RAY)
        with pytest.raises(am.AMError):
            m.march(precision="sliced")                     # the sliced operands carry no shortcut term
        # the compose of random patterns against the oracle's region-wise maps
        S = rng.integers(0, 2, size=(64, mlp.N)).astype(np.uint8)
        keys = np.zeros((64, (mlp.N + 63) // 64), dtype=np.uint64)
        for i, s in enumerate(S):
            for k in np.flatnonzero(s):
                keys[i, k >> 6] |= np.uint64(1) << np.uint64(k & 63)
        with pytest.raises(am.AMError):
            m.compose(nid, keys, "mixed")
        rows, _ = m.compose(nid, keys, "fp64")
        # sphere tracing uses the shortcut in its forward pass and gradient: its seeds lie on the
        # surface, in the oracle's cells
        starts = np.array([[1.2, 0.1, -0.2], [-0.3, 1.1, 0.4], [0.2, -0.4, -1.2], [0.9, 0.9, 0.9]])
        m.reset()
        _, pts = m.seed_sphere_trace(nid, starts, eta=1.0, max_steps=64, eps=1e-12)
    worst = 0.0
    for i, s in enumerate(S):
        A, aF = arch.res_compose(net, s)
        ref = np.vstack([(1.0 - 2.0 * s)[:, None] * A, aF[None, :]])
        worst = max(worst, float(np.abs(rows[i] - ref).max() / (1.0 + np.abs(ref).max())))
    print(f"\nresidual compose: max rel err {worst:.2e}")
    assert worst <= 1e-12
    ok = ~np.isnan(pts[:, 0])
    assert ok.sum() >= 3
    for p in pts[ok]:
        _, F = arch.res_forward(net, p)
        assert abs(F) < 1e-9
