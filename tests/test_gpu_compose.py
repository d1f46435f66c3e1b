"""The compose step alone (Lemma 1, Cor. 1, Eq. 10) through am_compose, against the oracle's
compose, in the four precisions.  FP64 agrees to rounding; the double-float rows lie within
their rigorous bounds; the split-BF16 tensor-core rows lie within their estimates; the sliced
tensor-core rows (error-free digit products) agree to FP64-class rounding.  Needs a GPU."""
import numpy as np
import pytest

from synth import decoder_net, proposal_target_net, sphere_net, tiny_net

pytestmark = pytest.mark.gpu
X_RAY = np.array([[1.0, 0.0, 0.0]])


def _keys_from_states(S, N):
    kw = (N + 63) // 64
    K = np.zeros((len(S), kw), dtype=np.uint64)
    for i, s in enumerate(S):
        for k in np.flatnonzero(s):
            K[i, k >> 6] |= np.uint64(1) << np.uint64(k & 63)
    return K


def _march_states(am, mlp, n, max_neurons, max_width):
    """Patterns of real cells: the first n cells of a march."""
    with am.Mesher(max_cells=1 << 16, max_neurons=max_neurons, max_width=max_width) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, np.zeros((1, 3)), X_RAY)
        m.march(max_cells=n)
        keys = m.get_mesh(nid).face_keys
    bits = np.unpackbits(keys.view(np.uint8), axis=1, bitorder="little")[:, :mlp.N]
    return bits.astype(np.uint8)


NETS = [
    ("tiny", lambda: tiny_net((8, 8), 11), 64, 32),
    ("sphere64x4", lambda: sphere_net(), 256, 64),
    ("decoder24x6", lambda: decoder_net(width=24, depth=6, latent_dim=9, skip_layer=3, seed=7, sigma=0.05), 256, 32),
    ("proposal256x8", lambda: proposal_target_net(), 2048, 256),
    ("decoder512x8", lambda: decoder_net(), 4096, 512),
]


@pytest.mark.parametrize("name,make,max_n,max_w", NETS)
def test_compose_matches_oracle(oracle_mod, name, make, max_n, max_w):
    import paper_2106_10031_gb300 as am
    mlp = make()
    net = oracle_mod.OracleNet(mlp)
    rng = np.random.default_rng(3)
    # random patterns (Lemma 1 holds for every pattern) and patterns of real cells
    S = np.concatenate([rng.integers(0, 2, (6, mlp.N)).astype(np.uint8),
                        _march_states(am, mlp, 10, max_n, max_w)[:10]])
    keys = _keys_from_states(S, mlp.N)
    ref = []
    for s in S:
        A, aF = net.compose(s)
        sg = (1.0 - 2.0 * s)[:, None]
        ref.append(np.vstack([sg * A, aF[None, :]]))
    ref = np.asarray(ref)
    scale = 1.0 + np.abs(ref).max(axis=2)
    with am.Mesher(max_cells=1 << 10, max_neurons=max_n, max_width=max_w) as m:
        nid = m.load_mlp(mlp)
        r64, _ = m.compose(nid, keys, "fp64")
        rdf, edf = m.compose(nid, keys, "mixed")
        rtc, etc = m.compose(nid, keys, "tensor")
        rsl, esl = m.compose(nid, keys, "sliced")
    err64 = np.abs(r64 - ref).max(axis=2) / scale
    assert err64.max() < 1e-11, err64.max()
    # sliced: every digit product and its FP32 accumulation is exact, so only the digits beyond
    # the eighth plane are lost, about 2^-48 of the row and column scales per term
    errsl = np.abs(rsl - ref).max(axis=2) / scale
    print(f"\n{name}: sliced max err {errsl.max():.2e} (fp64 {err64.max():.2e})")
    assert errsl.max() < 1e-11, errsl.max()
    assert np.all(esl == 0.0)
    # double-float: the l1 error of each row's 4 coefficients is within its rigorous bound
    # (plus the oracle's own FP64 rounding)
    l1 = np.abs(rdf - ref).sum(axis=2)
    assert np.all(l1 <= edf + 1e-12 * scale), (l1 - edf).max()
    # tensor cores: within the estimate on every row
    l1t = np.abs(rtc - ref).sum(axis=2)
    ratio = l1t / np.maximum(etc, 1e-30)
    rel = l1t / np.abs(ref).sum(axis=2).clip(1e-30)
    deep = ratio[:, mlp.widths[0]:]                  # rows of the tensor-core layers and a_F
    print(f"\n{name}: fp64 {err64.max():.1e}; mixed max err/bound {(l1 / np.maximum(edf, 1e-30)).max():.2e}; "
          f"tensor max rel {rel.max():.1e}, layers >= 2: max err/estimate {deep.max():.3f}, "
          f"p99 {np.quantile(deep, 0.99):.3f}, median {np.median(deep):.4f}; "
          f"median estimate (rel) {np.median(etc[:, mlp.widths[0]:] / np.abs(ref).sum(axis=2)[:, mlp.widths[0]:].clip(1e-30)):.1e}")
    assert np.all(l1t <= etc + 1e-12 * scale), ratio.max()


def test_march_refuses_tensor_rows(am_mod=None):
    # the march certifies every sign test; estimated rows cannot do that
    import paper_2106_10031_gb300 as am
    with am.Mesher(max_cells=1 << 10, max_neurons=64, max_width=32) as m:
        nid = m.load_mlp(tiny_net((8, 8), 11))
        m.seed(nid, np.zeros((1, 3)), X_RAY / 1.0)
        with pytest.raises(am.AMError) as e:
            m.march(precision="tensor")
        assert e.value.status == 1               # AM_ERR_INVALID_ARG


@pytest.mark.parametrize("tile_cells", [32, 16, 8])
def test_sliced_compose_batches_and_ragged_shapes(oracle_mod, tile_cells):
    # widths that fill no tile exactly, a skip layer with a latent, and more patterns than one
    # batch of the sliced compose (4096 cells): ragged rows, columns, K chunks and batches
    import paper_2106_10031_gb300 as am
    mlp = decoder_net(width=72, depth=5, latent_dim=5, skip_layer=3, seed=17, sigma=0.05)
    net = oracle_mod.OracleNet(mlp)
    rng = np.random.default_rng(5)
    n = 4096 + 37
    S = rng.integers(0, 2, (n, mlp.N)).astype(np.uint8)
    S[:3] = 0                                            # all neurons off: Z_l = C_l
    S[3:6] = 1                                           # all on
    keys = _keys_from_states(S, mlp.N)
    with am.Mesher(max_cells=1 << 10, max_neurons=512, max_width=128) as m:
        nid = m.load_mlp(mlp)
        m.set_tuning(compose_tile_cells=tile_cells)
        rsl, _ = m.compose(nid, keys, "sliced")
    worst = 0.0
    for i in list(range(8)) + list(rng.choice(n, 120, replace=False)) + list(range(n - 8, n)):
        A, aF = net.compose(S[i])
        sg = (1.0 - 2.0 * S[i])[:, None]
        ref = np.vstack([sg * A, aF[None, :]])
        err = np.abs(rsl[i] - ref).max(axis=1) / (1.0 + np.abs(ref).max(axis=1))
        worst = max(worst, err.max())
    print(f"\nsliced, {tile_cells} cells per tile: max err {worst:.2e} over 136 of {n} patterns")
    assert worst < 1e-11


def test_autotune_compose_and_tile_shapes_agree_bitwise(oracle_mod, tmp_path):
    # every tile shape sums the same exact digit products: the rows agree bit for bit; the
    # autotuner times each shape, keeps the fastest and caches its choice per net shape
    import paper_2106_10031_gb300 as am
    mlp = proposal_target_net()
    rng = np.random.default_rng(9)
    keys = _keys_from_states(rng.integers(0, 2, (700, mlp.N)).astype(np.uint8), mlp.N)
    cache = str(tmp_path / "tune.json")
    with am.Mesher(max_cells=1 << 10, max_neurons=2048, max_width=256) as m:
        nid = m.load_mlp(mlp)
        rows = {}
        for t in (0, 32, 16, 8):
            m.set_tuning(compose_tile_cells=t)
            rows[t], _ = m.compose(nid, keys, "sliced")
        assert all(np.array_equal(rows[t], rows[8]) for t in (0, 16, 32))
        res = m.autotune_compose(nid, keys, reps=3, cache=cache)
        assert not res["cached"] and res["compose_tile_cells"] in (0, 8, 16, 32)
        assert sorted(c["compose_tile_cells"] for c in res["candidates"]) == [0, 8, 16, 32]
        assert all(c["ms"] > 0 for c in res["candidates"])
        assert m.get_tuning()["compose_tile_cells"] == res["compose_tile_cells"]
        again = m.autotune_compose(nid, keys, cache=cache)
        assert again["cached"] and again["compose_tile_cells"] == res["compose_tile_cells"]
        with pytest.raises(am.AMError):
            m.set_tuning(compose_tile_cells=12)
        print(f"\nautotune: {res}")


def test_sliced_compose_edge_cases(oracle_mod):
    # one pattern; no pattern; a fan-in beyond the exact-accumulation limit (1638) is refused,
    # by am_compose and by the march, instead of being computed inexactly
    import paper_2106_10031_gb300 as am
    from synth.nets import MLP
    mlp = tiny_net((8, 8), 11)
    net = oracle_mod.OracleNet(mlp)
    s = np.random.default_rng(2).integers(0, 2, (1, mlp.N)).astype(np.uint8)
    with am.Mesher(max_cells=1 << 10, max_neurons=64, max_width=32) as m:
        nid = m.load_mlp(mlp)
        rows, _ = m.compose(nid, _keys_from_states(s, mlp.N), "sliced")
        A, aF = net.compose(s[0])
        ref = np.vstack([(1.0 - 2.0 * s[0])[:, None] * A, aF[None, :]])
        assert np.abs(rows[0] - ref).max() / (1.0 + np.abs(ref).max()) < 1e-11
        empty, _ = m.compose(nid, np.zeros((0, 1), dtype=np.uint64), "sliced")
        assert empty.shape[0] == 0
    rng = np.random.default_rng(3)
    wide = MLP(weights=[rng.normal(0, 0.5, (1700, 3)), rng.normal(0, 0.03, (8, 1700))],
               biases=[np.zeros(1700), np.zeros(8)], w_out=np.ones(8), b_out=-0.5, name="fanin1700")
    with am.Mesher(max_cells=1 << 10, max_neurons=2048, max_width=1700) as m:
        nid = m.load_mlp(wide)
        keys = _keys_from_states(rng.integers(0, 2, (2, wide.N)).astype(np.uint8), wide.N)
        with pytest.raises(am.AMError) as e:
            m.compose(nid, keys, "sliced")
        assert e.value.status == 1                          # AM_ERR_INVALID_ARG
        r64, _ = m.compose(nid, keys, "fp64")               # the other precisions still work
        assert np.isfinite(r64).all()
        with pytest.raises(am.AMError) as e:                 # refused before any work
            m.march(precision="sliced")
        assert e.value.status == 1
        with pytest.raises(am.AMError):
            m.set_tuning(compose_tile_cells=24)
