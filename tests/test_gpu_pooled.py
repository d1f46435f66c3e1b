"""A final max pooling over sub-networks on the device (Sec. 5.2, the paper's local-decoder
form): F = max_i F_i over M heads.  A cell is a unit pattern and the pooled index j (one-hot in
the device key's last M bits, j << N_units in the oracle's key); its system gains the pooling
rows a_F(i) - a_F(j) as planes N_units + i, its face lies on a_F(j), and crossing pooling plane
N_units + i moves the maximum to i.  The GPU mesh must be the oracle's (oracle/arch.py MaxPool)
face for face; its assembled vertices must join exactly the corners at one point (pooling
planes named by their pair of heads), and the closed surface must have Euler characteristic 2.
Needs a GPU."""
import numpy as np
import pytest

from oracle import arch
from synth import pooled_net
from tests import parity

pytestmark = pytest.mark.gpu
X_RAY = np.array([[1.0, 0.0, 0.0]])
ORIGIN = np.zeros((1, 3))


def to_pool(mlp):
    """The oracle's MaxPool of the sub-networks that pooled_net lays side by side."""
    w, M = mlp.meta["subnet_width"], len(mlp.heads)
    subs = []
    for i in range(M):
        sl = slice(i * w, (i + 1) * w)
        Ws = [mlp.weights[0][sl]] + [W[sl, sl] for W in mlp.weights[1:]]
        subs.append(arch.ResNet(Ws, [b[sl] for b in mlp.biases], mlp.heads[i][0][sl], mlp.heads[i][1], {}, mlp.slope))
    return arch.MaxPool(subs)


def unit_order(mlp):
    """perm[u] = the oracle's id of device unit u: the device numbers units layer by layer (the
    sub-networks side by side within a layer), the oracle's MaxPool sub-network by
    sub-network (each in layer order)."""
    w, M, L = mlp.meta["subnet_width"], len(mlp.heads), mlp.L
    perm = np.zeros(mlp.N, dtype=np.int64)
    for l in range(L):
        for i in range(M):
            for k in range(w):
                perm[l * M * w + i * w + k] = i * L * w + l * w + k
    return perm


def oracle_keyed(mesh, mlp):
    """The GPU mesh in the oracle's numbering: unit ids permuted (unit_order), and the one-hot
    pooled index j as j << N_units in the key."""
    from paper_2106_10031_gb300.mesher import Mesh
    n_units, M = mlp.N, len(mlp.heads)
    perm = unit_order(mlp)
    kw = (n_units + 6 + 63) // 64
    keys = np.zeros((mesh.n_faces, kw), dtype=np.uint64)
    for i in range(mesh.n_faces):
        k = parity._key_int(mesh.face_keys[i])
        onehot = k >> n_units
        assert onehot and onehot & (onehot - 1) == 0 and onehot < (1 << M), "pooled index not one-hot"
        v = (onehot.bit_length() - 1) << n_units
        for u in range(n_units):
            if (k >> u) & 1:
                v |= 1 << int(perm[u])
        keys[i] = np.frombuffer(v.to_bytes(8 * kw, "little"), dtype=np.uint64)
    e = mesh.edge_planes.astype(np.int64)
    e = np.where(e < n_units, perm[np.minimum(e, n_units - 1)], e).astype(np.int32)
    return Mesh(mesh.xyz, mesh.face_offsets, mesh.face_vertices, e, keys, mesh.n_open_faces)


def check_assembly(mesh, closed=True):
    """Distinct vertex indices are distinct points (the faces' coordinates, taken through their
    indices, are compared with the oracle's separately), and a closed surface has V - E + F = 2."""
    o, fv, xyz = mesh.face_offsets, mesh.face_vertices, mesh.xyz
    seen = {}
    for v, p in enumerate(np.round(xyz / 1e-9).astype(np.int64)):
        seen.setdefault(tuple(p), []).append(v)
    dup = [vs for vs in seen.values() if len(vs) > 1]
    assert not dup, f"{len(dup)} points carry more than one vertex index"
    edges = set()
    for i in range(mesh.n_faces):
        idx = fv[o[i]:o[i + 1]]
        for j in range(len(idx)):
            a, b = int(idx[j - 1]), int(idx[j])
            edges.add((min(a, b), max(a, b)))
    chi = len(xyz) - len(edges) + mesh.n_faces
    if closed:
        assert chi == 2, chi
    return chi


NETS = [lambda: pooled_net(seed=62, count=4, width=8, depth=3),
        lambda: pooled_net(seed=62, count=4, width=8, depth=4)]


@pytest.mark.parametrize("make", NETS)
@pytest.mark.parametrize("precision,schedule", [("fp64", "persistent"), ("fp64", "levels"), ("mixed", "persistent")])
def test_pooled_mesh_matches_oracle(oracle_mod, make, precision, schedule):
    import paper_2106_10031_gb300 as am
    from paper_2106_10031_gb300.mesher import device_N
    mlp = make()
    M, nU = len(mlp.heads), mlp.N
    pool = to_pool(mlp)
    ref = arch.march(pool, [arch.seed_ray(pool, ORIGIN[0], X_RAY[0])])
    assert ref.faces and not ref.failed
    with am.Mesher(max_cells=1 << 17, max_neurons=max(64, device_N(mlp)), max_width=max(mlp.widths)) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, ORIGIN, X_RAY)
        m.march(precision=precision, schedule=schedule)
        mesh = m.get_mesh(nid)
        st = m.stats()
    got = oracle_keyed(mesh, mlp)
    ref_faces = {f.key: f for f in ref.faces}
    gf = parity.gpu_faces(got)
    assert set(gf) == set(ref_faces), (len(set(gf) - set(ref_faces)), len(set(ref_faces) - set(gf)))
    worst = 0.0
    for k, f in ref_faces.items():
        e_g, v_g, _ = gf[k]
        assert f.edges == e_g, (hex(k), f.edges, e_g)
        worst = max(worst, float((np.linalg.norm(f.verts - v_g, axis=1) / np.maximum(1.0, np.linalg.norm(f.verts, axis=1))).max()))
    n_pool = sum(1 for f in ref.faces for e in f.edges if nU <= e < nU + M)
    js = {f.key >> nU for f in ref.faces}
    chi = check_assembly(mesh, closed=mesh.n_open_faces == 0)
    print(f"\n{mlp.name} {precision}/{schedule}: {len(gf)} faces, {n_pool} pooling edges, pooled indices {sorted(js)}, "
          f"max rel vertex err {worst:.2e}, chi {chi}")
    assert worst <= 1e-9 and st["degenerate"] == 0
    assert n_pool > 0 and len(js) == M
    assert mesh.n_open_faces == 0
    if precision == "mixed":
        assert st["refined_cells"] == st["cells"]          # pooled nets march in FP64


def test_pooled_compose_and_triggers(oracle_mod):
    # the pooled net's compose against the oracle's subcell rows, and sphere tracing with the
    # gradient of the pooled head: its seeds lie on the surface
    import paper_2106_10031_gb300 as am
    from paper_2106_10031_gb300.mesher import device_N
    mlp = pooled_net(seed=62, count=4, width=8, depth=4)
    M, nU = len(mlp.heads), mlp.N
    pool = to_pool(mlp)
    rng = np.random.default_rng(9)
    S = rng.integers(0, 2, size=(32, nU)).astype(np.uint8)
    J = rng.integers(0, M, size=32)
    N = device_N(mlp)
    keys = np.zeros((32, (N + 63) // 64), dtype=np.uint64)
    for i, (s, j) in enumerate(zip(S, J)):
        for k in list(np.flatnonzero(s)) + [nU + int(j)]:
            keys[i, k >> 6] |= np.uint64(1) << np.uint64(k & 63)
    with am.Mesher(max_cells=1 << 16, max_neurons=max(64, N), max_width=max(mlp.widths)) as m:
        nid = m.load_mlp(mlp)
        rows, _ = m.compose(nid, keys, "fp64")
        # |grad F| is about 3 here (not a distance function): the walk takes a fifth of each step
        starts = np.array([[1.2, 0.1, -0.2], [-0.3, 1.1, 0.4], [0.2, -0.4, -1.2], [0.9, 0.9, 0.9]])
        _, pts = m.seed_sphere_trace(nid, starts, eta=0.2, max_steps=64, eps=1e-12)
    worst = 0.0
    perm = unit_order(mlp)
    for i, (s, j) in enumerate(zip(S, J)):
        s_or = np.zeros(nU, dtype=np.uint8)
        s_or[perm] = s                                      # the oracle's pattern of device pattern s
        C, ids, aF = pool.cell_rows(s_or, int(j), box=1.5)
        inv = np.empty(nU, dtype=np.int64)
        inv[perm] = np.arange(nU)                           # oracle unit id -> device unit id
        want = np.zeros((N + 1, 4))
        for r, pid in zip(C, ids):
            if pid < nU:
                want[inv[pid]] = r
            elif pid < N:
                want[pid] = r
        want[N] = aF
        worst = max(worst, float(np.abs(rows[i] - want).max() / (1.0 + np.abs(want).max())))
    print(f"\npooled compose: max rel err {worst:.2e}")
    assert worst <= 1e-12
    ok = ~np.isnan(pts[:, 0])
    assert ok.sum() >= 2                                # two starts reach |F| < 1e-12 in 64 steps
    for p in pts[ok]:
        assert abs(pool.forward(p)[2]) < 1e-9
