"""The rank-1 neighbour compose (Cor. 1 across one flipped neuron; Alg. 1 step 10) on the tensor
cores: the rows of real neighbour cells from their parents' rows against the oracle's compose of
the neighbours' patterns, flips in every layer; and the sliced march that composes most cells
this way against the same march composing every cell in full (identical faces, edge cycles and
vertices) and against the oracle.  Needs a GPU."""
import numpy as np
import pytest

from synth import decoder_net, proposal_target_net, sphere_net, tiny_net
from tests import parity

pytestmark = pytest.mark.gpu
X_RAY = np.array([[1.0, 0.0, 0.0]])
ORIGIN = np.zeros((1, 3))

NETS = [
    ("tiny", lambda: tiny_net((8, 8), 11), 64, 32),
    ("sphere64x4", lambda: sphere_net(), 256, 64),
    ("decoder24x6", lambda: decoder_net(width=24, depth=6, latent_dim=9, skip_layer=3, seed=7, sigma=0.05), 256, 32),
    ("proposal256x8", lambda: proposal_target_net(), 2048, 256),
    ("decoder512x8", lambda: decoder_net(), 4096, 512),
]


def _neighbour_pairs(am, mlp, max_n, max_w, per_layer=24, seed=0):
    """(parent key, flipped neuron) of real edges of a march's faces, up to per_layer flips in
    every hidden layer."""
    with am.Mesher(max_cells=1 << 16, max_neurons=max_n, max_width=max_w) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, ORIGIN, X_RAY)
        m.march(max_cells=4000)
        mesh = m.get_mesh(nid)
    rng = np.random.default_rng(seed)
    face = np.repeat(np.arange(mesh.n_faces), np.diff(mesh.face_offsets))
    e = mesh.edge_planes.astype(np.int64)
    inner = np.flatnonzero(e < mlp.N)
    bounds = np.cumsum([0] + mlp.widths)
    pick = []
    for l in range(mlp.L):
        cand = inner[(e[inner] >= bounds[l]) & (e[inner] < bounds[l + 1])]
        if len(cand):
            pick.extend(rng.choice(cand, min(per_layer, len(cand)), replace=False))
    pick = np.asarray(pick)
    kw = (mlp.N + 63) // 64                  # the context's keys may be wider than the net's
    return np.ascontiguousarray(mesh.face_keys[face[pick], :kw]), e[pick].astype(np.int32)


@pytest.mark.parametrize("name,make,max_n,max_w", NETS)
def test_rank1_rows_match_oracle(oracle_mod, name, make, max_n, max_w):
    import paper_2106_10031_gb300 as am
    mlp = make()
    keys, flips = _neighbour_pairs(am, mlp, max_n, max_w)
    with am.Mesher(max_cells=1 << 10, max_neurons=max_n, max_width=max_w) as m:
        nid = m.load_mlp(mlp)
        parent_rows, _ = m.compose(nid, keys, "sliced")
        rows = m.compose_neighbors(nid, keys, parent_rows, flips)
        # the children composed in full on the tensor cores, for comparison
        child_keys = keys.copy()
        for i, f in enumerate(flips):
            child_keys[i, f >> 6] ^= np.uint64(1) << np.uint64(f & 63)
        full, _ = m.compose(nid, child_keys, "sliced")
    net = oracle_mod.OracleNet(mlp)
    bits = np.unpackbits(child_keys.view(np.uint8), axis=1, bitorder="little")[:, :mlp.N].astype(np.uint8)
    ref = []
    for s in bits:
        A, aF = net.compose(s)
        ref.append(np.vstack([(1.0 - 2.0 * s)[:, None] * A, aF[None, :]]))
    ref = np.asarray(ref)
    scale = 1.0 + np.abs(ref).max(axis=2)
    err = np.abs(rows - ref).max(axis=2) / scale
    err_full = np.abs(full - ref).max(axis=2) / scale
    layers = np.searchsorted(np.cumsum(mlp.widths), flips, side="right") + 1
    print(f"\n{name}: rank-1 max err {err.max():.2e} (full sliced {err_full.max():.2e}), flips in layers "
          f"{sorted(set(layers.tolist()))}, {len(flips)} children")
    assert set(layers.tolist()) == set(range(1, mlp.L + 1))      # a flip in every layer, the last included
    assert err.max() < 1e-11, err.max()


@pytest.mark.parametrize("period", [2, 8, 1000])
def test_rank1_march_equals_full_march(oracle_mod, period):
    # the sphere net's whole mesh with the rank-1 compose (a full compose every `period`
    # generations; 1000 lets the chains run the whole depth) against every cell composed in full
    import paper_2106_10031_gb300 as am
    mlp = sphere_net()
    meshes, stats = {}, {}
    with am.Mesher(max_cells=1 << 17, max_neurons=256, max_width=64) as m:
        nid = m.load_mlp(mlp)
        for p in (1, period):
            m.set_tuning(rank1_period=p)
            m.reset()
            m.seed(nid, ORIGIN, X_RAY)
            m.march(precision="sliced")
            meshes[p], stats[p] = m.get_mesh(nid), m.stats()
    full, r1 = parity.gpu_faces(meshes[1]), parity.gpu_faces(meshes[period])
    assert set(full) == set(r1)
    assert all(full[k][0] == r1[k][0] for k in full)
    worst = max(float(np.abs(full[k][1] - r1[k][1]).max()) for k in full)
    print(f"\nperiod {period}: {len(full)} faces, max vertex difference {worst:.2e}, compose "
          f"{stats[period]['ms_compose']:.1f} ms vs {stats[1]['ms_compose']:.1f} ms in full")
    assert worst < 1e-9 and stats[period]["degenerate"] == 0
    net, ref = oracle_mod.mesh_from_rays(mlp, ORIGIN, X_RAY)
    parity.compare(ref, meshes[period], mlp.N, rtol=1e-9)
