"""Parity of the CUDA path (through the C ABI) with the CPU oracle.  Needs a GPU."""
import numpy as np
import pytest

from synth import batch_nets, decoder_net, octahedron, polytope_max_of_planes, sphere_net, tiny_net
from tests import parity

pytestmark = pytest.mark.gpu

RAY = np.array([[1.0, 0.37, 0.21]]) / np.linalg.norm([1.0, 0.37, 0.21])
X_RAY = np.array([[1.0, 0.0, 0.0]])


@pytest.fixture(scope="module")
def am():
    import paper_2106_10031_gb300 as am_mod
    return am_mod


# sliced: the compose on the tensor cores as exact digit-plane products (FP64-class rows), the
# clip in FP64; it always runs the level schedule
MODES = [("fp64", "persistent", 1e-9), ("mixed", "persistent", 1e-5), ("fp64", "levels", 1e-9),
         ("mixed", "levels", 1e-5), ("sliced", "levels", 1e-9)]


def _both(oracle_mod, am, mlp, dirs, R=2.0, **kw):
    net, ref = oracle_mod.mesh_from_rays(mlp, np.zeros((len(dirs), 3)), dirs, R)
    with am.Mesher(max_cells=kw.pop("max_cells", 1 << 18), max_neurons=max(64, mlp.N),
                   max_width=max(mlp.widths)) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, np.zeros((len(dirs), 3)), dirs, R)
        m.march(**kw)
        mesh = m.get_mesh(nid)
        st = m.stats()
    return net, ref, mesh, st


@pytest.mark.parametrize("precision,schedule,rtol", MODES)
@pytest.mark.parametrize("make,dirs", [
    (octahedron, RAY),
    (polytope_max_of_planes, X_RAY),
    (lambda: tiny_net((8, 8), 11), RAY),
    (lambda: tiny_net((6, 5, 4), 12), RAY),
    (lambda: decoder_net(width=24, depth=6, latent_dim=9, skip_layer=3, seed=7, sigma=0.05), X_RAY),
])
def test_parity_small(oracle_mod, am, make, dirs, precision, schedule, rtol):
    mlp = make()
    net, ref, mesh, st = _both(oracle_mod, am, mlp, dirs, precision=precision, schedule=schedule)
    assert not ref.failed
    r = parity.compare(ref, mesh, mlp.N, rtol=rtol)
    assert st["degenerate"] == 0 == ref.degenerate
    assert st["faces"] == r["faces"]
    assert mesh.n_open_faces == ref.open_faces()


@pytest.mark.parametrize("precision,schedule,rtol", MODES)
def test_parity_sphere_net_full(oracle_mod, am, precision, schedule, rtol):
    # the 3-[64]x4-1 workload at full size, every face compared
    mlp = sphere_net()
    net, ref, mesh, st = _both(oracle_mod, am, mlp, X_RAY, precision=precision, schedule=schedule)
    r = parity.compare(ref, mesh, mlp.N, rtol=rtol)
    assert r["faces"] > 40000 and st["degenerate"] == 0 and mesh.n_open_faces == 0
    print(f"{precision}/{schedule}: max rel vertex err {r['max_rel_vertex_err']:.2e}, refined {st['refined_cells']}, "
          f"close calls {st['close_calls']}, fixups {st['fixups']}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parity_multi_seed_multi_component(oracle_mod, am, precision):
    # many rays, some landing in the same cell, on a net with several surface components
    mlp = tiny_net((6, 5, 4), 12)
    rng = np.random.default_rng(5)
    d = rng.normal(size=(64, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    net, ref, mesh, st = _both(oracle_mod, am, mlp, d, precision=precision)
    parity.compare(ref, mesh, mlp.N, rtol=1e-5)


def test_parity_two_nets_one_march(oracle_mod, am):
    nets = [sphere_net(seed=21, width=32, depth=4, sigma=0.05), tiny_net((8, 8), 11)]
    refs = [oracle_mod.mesh_from_rays(n, np.zeros((1, 3)), RAY)[1] for n in nets]
    with am.Mesher(max_cells=1 << 18, max_neurons=256, max_width=64) as m:
        ids = [m.load_mlp(n) for n in nets]
        for i in ids:
            m.seed(i, np.zeros((1, 3)), RAY)
        m.march()
        for i, n, r in zip(ids, nets, refs):
            parity.compare(r, m.get_mesh(i), n.N, rtol=1e-9)


def test_device_mesh_view_matches_the_copy(am):
    """am_get_mesh_device hands out views of the context's buffers: for every net of a
    two-net march they equal what am_get_mesh copies out, bit for bit, and a second net's
    view leaves the first one's intact."""
    import torch
    nets = [sphere_net(seed=21, width=32, depth=4, sigma=0.05), tiny_net((8, 8), 11)]
    with am.Mesher(max_cells=1 << 18, max_neurons=256, max_width=64) as m:
        with pytest.raises(am.AMError):
            m.get_mesh_device(0)
        ids = [m.load_mlp(n) for n in nets]
        for i in ids:
            m.seed(i, np.zeros((1, 3)), RAY)
        m.march()
        views = [m.get_mesh_device(i) for i in ids]
        for i, v in zip(ids, views):
            host = m.get_mesh(i)
            assert v["xyz"].is_cuda and v["xyz"].dtype == torch.float64
            np.testing.assert_array_equal(v["xyz"].cpu().numpy(), host.xyz)
            np.testing.assert_array_equal(v["face_offsets"].cpu().numpy(), host.face_offsets)
            np.testing.assert_array_equal(v["face_vertices"].cpu().numpy(), host.face_vertices)
            np.testing.assert_array_equal(v["edge_planes"].cpu().numpy(), host.edge_planes)
            np.testing.assert_array_equal(v["face_keys"].cpu().numpy().view(np.uint64), host.face_keys)
            assert host.n_faces > 0 and int(v["face_offsets"][0]) == 0


@pytest.mark.parametrize("schedule", ["persistent", "levels"])
def test_resume_after_max_cells(oracle_mod, am, schedule):
    mlp = sphere_net(seed=21, width=32, depth=4, sigma=0.05)
    net, ref = oracle_mod.mesh_from_rays(mlp, np.zeros((1, 3)), RAY)
    with am.Mesher(max_cells=1 << 17, max_neurons=128, max_width=32) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, np.zeros((1, 3)), RAY)
        st = m.march(max_cells=500, schedule=schedule)
        assert st == 7                      # AM_INCOMPLETE
        while m.march(max_cells=500, schedule=schedule) == 7:
            pass
        parity.compare(ref, m.get_mesh(nid), mlp.N, rtol=1e-9)


def test_persistent_with_few_blocks(oracle_mod, am):
    # a grid smaller than the machine: blocks wait for work published by other blocks
    mlp = sphere_net(seed=21, width=32, depth=4, sigma=0.05)
    net, ref, mesh, st = _both(oracle_mod, am, mlp, RAY, grid_blocks=3, precision="mixed")
    parity.compare(ref, mesh, mlp.N, rtol=1e-5)


def test_capacity_error_is_reported(am):
    mlp = sphere_net()
    with am.Mesher(max_cells=1000, max_neurons=256, max_width=64) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, np.zeros((1, 3)), X_RAY)
        with pytest.raises(am.AMError) as e:
            m.march()
        assert e.value.status == 3           # AM_ERR_CAPACITY


def test_seed_without_sign_change(am):
    with am.Mesher(max_cells=1024, max_neurons=256, max_width=64) as m:
        nid = m.load_mlp(sphere_net())
        with pytest.raises(am.AMError) as e:
            m.seed(nid, np.zeros((1, 3)), X_RAY, R=0.05)
        assert e.value.status == 5           # AM_ERR_NO_SEED_CELL


def test_seed_matches_oracle(oracle_mod, am):
    # the device bisection lands in the oracle's seed cell
    for mlp in (sphere_net(), decoder_net(width=24, depth=6, latent_dim=9, skip_layer=3, seed=7, sigma=0.05)):
        net, ref = oracle_mod.mesh_from_rays(mlp, np.zeros((1, 3)), X_RAY, max_cells=1)
        with am.Mesher(max_cells=4096, max_neurons=256, max_width=64) as m:
            nid = m.load_mlp(mlp)
            m.seed(nid, np.zeros((1, 3)), X_RAY)
            m.march(max_cells=1)
            mesh = m.get_mesh(nid)
        assert mesh.n_faces == 1
        assert parity._key_int(mesh.face_keys[0]) == ref.seeds[0][0]


def test_sliced_march_with_a_wider_context(oracle_mod, am):
    # the context's key width (max_neurons) larger than the net's: the march's cell keys are
    # strided by the context, the compose's by the net
    mlp = sphere_net(seed=21, width=32, depth=4, sigma=0.05)
    net, ref = oracle_mod.mesh_from_rays(mlp, np.zeros((1, 3)), RAY)
    with am.Mesher(max_cells=1 << 17, max_neurons=512, max_width=64) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, np.zeros((1, 3)), RAY)
        m.march(precision="sliced")
        parity.compare(ref, m.get_mesh(nid), mlp.N, rtol=1e-9)


def test_sliced_march_needs_one_net(am):
    # the tensor-core compose works on batches of one net's cells
    with am.Mesher(max_cells=1 << 12, max_neurons=256, max_width=64) as m:
        for n in (sphere_net(seed=21, width=32, depth=4, sigma=0.05), tiny_net((8, 8), 11)):
            i = m.load_mlp(n)
            m.seed(i, np.zeros((1, 3)), RAY)
        with pytest.raises(am.AMError) as e:
            m.march(precision="sliced")
        assert e.value.status == 1           # AM_ERR_INVALID_ARG


def test_march_autotuner_times_every_path(am):
    # every precision x schedule gives the oracle's mesh, so the fastest one is a free choice
    mlp = sphere_net(seed=21, width=32, depth=4, sigma=0.05)
    with am.Mesher(max_cells=1 << 17, max_neurons=128, max_width=32) as m:
        nid = m.load_mlp(mlp)
        res = m.autotune_march(nid, np.zeros((1, 3)), RAY, max_cells=5000, reps=1)
        tried = {(c["precision"], c["schedule"]) for c in res["candidates"]}
        assert tried == {("fp64", "persistent"), ("mixed", "persistent"), ("fp64", "levels"), ("mixed", "levels"),
                         ("sliced", "levels")}
        assert all(c["ms"] > 0 for c in res["candidates"])
        assert (res["precision"], res["schedule"]) in tried
        assert m.stats()["cells"] == 0                   # the tuner leaves no cells behind
        m.seed(nid, np.zeros((1, 3)), RAY)
        m.march(precision=res["precision"], schedule=res["schedule"])
        assert m.get_mesh(nid).n_faces > 10000
        print(f"\nmarch autotuner: {res}")


@pytest.mark.parametrize("make,dirs", [
    (lambda: tiny_net((6, 5, 4), 12), RAY),
    (lambda: decoder_net(width=24, depth=6, latent_dim=9, skip_layer=3, seed=7, sigma=0.05), X_RAY),
])
def test_sliced_rows_with_the_plain_clip(oracle_mod, am, make, dirs):
    # tensor-core rows clipped by every cutting row (no candidates): the plain method's path
    mlp = make()
    net, ref, mesh, st = _both(oracle_mod, am, mlp, dirs, precision="sliced", candidates="none")
    parity.compare(ref, mesh, mlp.N, rtol=1e-9)
    assert st["degenerate"] == 0 and st["fixups"] == st["cells"]       # every face found by the check
