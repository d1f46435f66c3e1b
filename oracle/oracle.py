"""Plain FP64 CPU oracle for analytic marching (arXiv 2106.10031).

TEST INFRASTRUCTURE ONLY.  Imported by the test suite, by the smoke check and
by the benchmark's CPU-baseline leg; never by the library.  It shares no code
with the CUDA path: its per-cell arithmetic is the plain C in ``am_oracle.c``
(loaded with ctypes) and the marching loop below is a literal FIFO rendering
of Algorithm 1.

What it computes (the definition the CUDA path must reproduce):
  * the set of non-empty analytic faces (Eq. 12) reachable from the seed cells
    through shared edges (Alg. 1), each face clipped to the box [-B, B]^3;
  * per face: its cell key s (bit k = state of neuron k, layer order, Def. 2),
    its vertices in CCW order seen from +grad F (= a_F[0:3]) starting at the
    canonical vertex, and for each edge the id of the plane carrying it
    (neuron id < N, or N + {0..5} for the box faces +x,-x,+y,-y,+z,-z);
  * an assembled mesh whose vertices are identified by the combinatorial key
    (i, j, s with bits i and j cleared), i < j the two planes meeting there.

Readings of the paper taken here (the CUDA path takes the same ones):
  * biases kept, affine rows [a | a_0] (Sec. 2.2 omits them for notation);
  * a tie a_lk = 0 gives state 0 (Eq. 2);
  * unbounded cells/faces are clipped to the box [-B, B]^3 (Sec. 3.1 lets
    faces extend without bound);
  * vertex validity (Alg. 1 step 8) uses a distance tolerance delta; rows within
    delta of an accepted vertex are counted as degenerate events;
  * Alg. 2's starting boundary for a seed cell is the row whose in-plane line
    is nearest to the seed point; marched cells start from the switching plane
    and the midpoint of the switching edge (Sec. 4.2.1);
  * faces of area <= 1e-24 B^2 are dropped and counted (Sec. 3.1: a face exists
    when the plane meets the cell's interior);
  * seeds come from bisection along a ray (Sec. 4.3.2), stopped when both
    bracket ends share one cell, then the exact affine root in that cell;
  * the sphere-tracing trigger (Sec. 4.3.1) stops after a step budget or once
    |F| <= eps, then bisects a short segment along the gradient through its last
    point (trace_bracket); the random-pair trigger (Sec. 4.3.2) pairs the r-th
    positive sample with the r-th negative one (sign_pairs).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from collections import deque
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "am_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liborc.so")

DEFAULT_BOX = 1.5
DEFAULT_DELTA = 1e-10
N_BOX = 6

_lib = None


def build(force: bool = False) -> str:
    """Compile am_oracle.c into a shared library (plain gcc, portable flags)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str | None = None):
    """ctypes handle on the compiled oracle (the default build, or another build at ``path``)."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    lib = ctypes.CDLL(path or build())
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    lib.orc_forward.argtypes = [P, P, P, P, P]
    lib.orc_state.argtypes = [P, P, P, P, P]
    lib.orc_compose.argtypes = [P, P, P, P, P]
    lib.orc_cell_rows.argtypes = [P, P, P, D, P, P]
    lib.orc_pivot.argtypes = [I, P, P, I, P, D, I, P, P, P, P]
    lib.orc_nearest_line.argtypes = [I, P, P, P]
    lib.orc_seed_ray.argtypes = [P, P, P, P, D, I, P, P, P]
    lib.orc_sphere_trace.argtypes = [P, P, P, D, I, D, P, P, P, P]
    for f in ("orc_forward", "orc_state", "orc_compose", "orc_cell_rows", "orc_pivot",
              "orc_nearest_line", "orc_seed_ray", "orc_sphere_trace"):
        getattr(lib, f).restype = I
    if path is None:
        _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------------------------
# keys: a cell key is a Python int whose bit k is the state of neuron k (layer order)


def state_to_key(s: np.ndarray) -> int:
    s = np.asarray(s, dtype=np.uint8)
    b = np.packbits(s, bitorder="little")
    return int.from_bytes(b.tobytes(), "little")


def key_to_state(key: int, N: int) -> np.ndarray:
    nbytes = (N + 7) // 8
    b = np.frombuffer(key.to_bytes(nbytes, "little"), dtype=np.uint8)
    return np.unpackbits(b, bitorder="little")[:N].astype(np.uint8)


def key_to_words(key: int, W: int) -> np.ndarray:
    return np.frombuffer(key.to_bytes(8 * W, "little"), dtype=np.uint64).copy()


def words_to_key(w) -> int:
    return int.from_bytes(np.asarray(w, dtype=np.uint64).tobytes(), "little")


# --------------------------------------------------------------------------------------------


class OracleNet:
    """One MLP packed into the oracle's flat format."""

    def __init__(self, mlp, lib=None):
        self.mlp = mlp
        self.N = mlp.N
        desc = [mlp.L, mlp.in_dim, mlp.skip_layer] + list(mlp.widths)
        self.desc = np.asarray(desc, dtype=np.int32)
        parts = []
        for W, b in zip(mlp.weights, mlp.biases):
            parts += [np.ascontiguousarray(W, dtype=np.float64).ravel(), np.asarray(b, dtype=np.float64)]
        parts += [np.asarray(mlp.w_out, dtype=np.float64), np.array([mlp.b_out], dtype=np.float64)]
        if mlp.latent is not None:
            parts.append(np.asarray(mlp.latent, dtype=np.float64))
        self.prm = np.ascontiguousarray(np.concatenate(parts))
        self.lib = lib if lib is not None else load_library()

    # Eq. 1 and Def. 2
    def forward(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        pre = np.zeros(self.N)
        F = np.zeros(1)
        rc = self.lib.orc_forward(_p(self.desc), _p(self.prm), _p(x), _p(pre), _p(F))
        assert rc == 0
        return pre, float(F[0])

    def F(self, x) -> float:
        return self.forward(x)[1]

    def state(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        s = np.zeros(self.N, dtype=np.uint8)
        F = np.zeros(1)
        rc = self.lib.orc_state(_p(self.desc), _p(self.prm), _p(x), _p(s), _p(F))
        assert rc == 0
        return s

    # Cor. 1
    def compose(self, s):
        s = np.ascontiguousarray(s, dtype=np.uint8)
        A = np.zeros((self.N, 4))
        aF = np.zeros(4)
        rc = self.lib.orc_compose(_p(self.desc), _p(self.prm), _p(s), _p(A), _p(aF))
        assert rc == 0
        return A, aF

    # Eq. 10 + box rows
    def cell_rows(self, s, B=DEFAULT_BOX):
        s = np.ascontiguousarray(s, dtype=np.uint8)
        C = np.zeros((self.N + N_BOX, 4))
        aF = np.zeros(4)
        rc = self.lib.orc_cell_rows(_p(self.desc), _p(self.prm), _p(s), float(B), _p(C), _p(aF))
        assert rc == 0
        return C, aF

    # Sec. 4.3.2
    def seed_ray(self, o, d, R=2.0, max_halvings=200):
        o = np.ascontiguousarray(o, dtype=np.float64)
        d = np.ascontiguousarray(d, dtype=np.float64)
        x = np.zeros(3)
        s = np.zeros(self.N, dtype=np.uint8)
        it = np.zeros(1, dtype=np.int32)
        rc = self.lib.orc_seed_ray(_p(self.desc), _p(self.prm), _p(o), _p(d), float(R), int(max_halvings),
                                   _p(x), _p(s), _p(it))
        return rc, x, s, int(it[0])

    # Sec. 4.3.1
    def sphere_trace(self, x0, eta=1.0, max_steps=64, eps=1e-12):
        """Sphere-tracing walk from x0: (rc, last point, F there, gradient of its cell, steps)."""
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        x, g, F = np.zeros(3), np.zeros(3), np.zeros(1)
        t = np.zeros(1, dtype=np.int32)
        rc = self.lib.orc_sphere_trace(_p(self.desc), _p(self.prm), _p(x0), float(eta), int(max_steps), float(eps),
                                       _p(x), _p(F), _p(g), _p(t))
        return rc, x, float(F[0]), g, int(t[0])


def face_pivot(C, aF, start, x, delta=DEFAULT_DELTA, max_v=256, lib=None):
    """Alg. 2 on the rows C.  Returns (rc, V (nv x 3), pairs (nv x 2), ndeg)."""
    lib = lib if lib is not None else load_library()
    C = np.ascontiguousarray(C, dtype=np.float64)
    aF = np.ascontiguousarray(aF, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    V = np.zeros((max_v, 3))
    pairs = np.zeros((max_v, 2), dtype=np.int32)
    nv = np.zeros(1, dtype=np.int32)
    nd = np.zeros(1, dtype=np.int32)
    rc = lib.orc_pivot(int(C.shape[0]), _p(C), _p(aF), int(start), _p(x), float(delta), int(max_v),
                       _p(V), _p(pairs), _p(nv), _p(nd))
    n = int(nv[0])
    return rc, V[:n].copy(), pairs[:n].copy(), int(nd[0])


def nearest_line(C, aF, x, lib=None) -> int:
    lib = lib if lib is not None else load_library()
    C = np.ascontiguousarray(C, dtype=np.float64)
    aF = np.ascontiguousarray(aF, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return int(lib.orc_nearest_line(int(C.shape[0]), _p(C), _p(aF), _p(x)))


def face_allpairs(C, aF, delta=DEFAULT_DELTA):
    """Alg. 1 steps 6-9: solve Eq. 11 for every pair of rows, keep the valid solutions.

    An independent second clip (numpy, batched).  Returns (V (m x 3), pairs (m x 2)) with
    the vertices ordered by angle around their mean in the face plane (CCW seen from
    +a_F[0:3]); empty arrays when fewer than 3 valid vertices exist.
    """
    C = np.asarray(C, dtype=np.float64)
    M = C.shape[0]
    nrm = np.linalg.norm(C[:, :3], axis=1)
    I, J = np.triu_indices(M, 1)
    keep = (nrm[I] > 0) & (nrm[J] > 0)
    I, J = I[keep], J[keep]
    A = np.stack([C[I, :3], C[J, :3], np.broadcast_to(aF[:3], (len(I), 3))], axis=1)
    rhs = -np.stack([C[I, 3], C[J, 3], np.full(len(I), aF[3])], axis=1)
    det = np.linalg.det(A)
    ok = np.abs(det) > 0
    I, J, A, rhs = I[ok], J[ok], A[ok], rhs[ok]
    v = np.linalg.solve(A, rhs[..., None])[..., 0]
    finite = np.all(np.isfinite(v), axis=1)
    I, J, v = I[finite], J[finite], v[finite]
    safe = np.where(nrm > 0, nrm, 1.0)
    dist = (v @ C[:, :3].T + C[:, 3]) / safe            # (P, M)
    dist[:, nrm == 0] = np.where(C[nrm == 0, 3] > 0, np.inf, -np.inf)
    dist[np.arange(len(I)), I] = -np.inf
    dist[np.arange(len(J)), J] = -np.inf
    valid = np.all(dist <= delta, axis=1)
    V, P = v[valid], np.stack([I[valid], J[valid]], 1)
    if len(V) < 3:
        return np.zeros((0, 3)), np.zeros((0, 2), dtype=np.int64)
    n = aF[:3] / np.linalg.norm(aF[:3])
    c = V.mean(0)
    u = V[0] - c
    u -= n * (u @ n)
    u /= np.linalg.norm(u)
    w = np.cross(n, u)
    ang = np.arctan2((V - c) @ w, (V - c) @ u)
    o = np.argsort(ang, kind="stable")
    return V[o], P[o]


# --------------------------------------------------------------------------------------------
# faces and meshes


@dataclass
class Face:
    key: int
    edges: list            # plane id of the edge from vertex i to vertex i+1 (CCW)
    verts: np.ndarray      # (m, 3)
    aF: np.ndarray         # (4,)
    ndeg: int = 0

    def vertex_pair(self, i):
        m = len(self.edges)
        a, b = self.edges[i - 1 if i > 0 else m - 1], self.edges[i]
        return (min(a, b), max(a, b))

    def area(self) -> float:
        return 0.5 * float(np.linalg.norm(newell(self.verts)))


def newell(V: np.ndarray) -> np.ndarray:
    """Twice the vector area of the closed polygon V: the sum of V_i x V_{i+1}, taken about the
    first vertex (the sum is translation invariant), so that a face far smaller than its
    distance from the origin keeps its area instead of cancelling to zero."""
    D = V - V[0]
    return np.cross(D, np.roll(D, -1, axis=0)).sum(0)


def canonical_face(key: int, V: np.ndarray, edges: list, aF: np.ndarray, ndeg: int = 0) -> Face:
    """Orient CCW seen from +a_F[0:3] and rotate to start at the vertex whose (sorted) pair of
    planes is lexicographically smallest.  edges[i] is the plane of edge V[i] -> V[i+1]."""
    V = np.asarray(V, dtype=np.float64)
    m = len(edges)
    edges = list(int(e) for e in edges)
    if float(newell(V) @ aF[:3]) < 0.0:
        V = V[::-1].copy()
        edges = [edges[(m - 2 - j) % m] for j in range(m)]
    pairs = [(min(edges[j - 1], edges[j]), max(edges[j - 1], edges[j])) for j in range(m)]
    j0 = min(range(m), key=lambda j: pairs[j])
    V = np.roll(V, -j0, axis=0)
    edges = edges[j0:] + edges[:j0]
    return Face(key, edges, V, np.asarray(aF, dtype=np.float64), ndeg)


def face_from_pivot(key, V, pairs, aF, ndeg=0) -> Face:
    # vertex j lies between plane pairs[j,0] (walked before) and pairs[j,1] (walked after):
    # the edge V[j] -> V[j+1] is carried by pairs[j,1].
    return canonical_face(key, V, [int(p[1]) for p in pairs], aF, ndeg)


@dataclass
class Mesh:
    N: int
    box: float
    faces: list = field(default_factory=list)
    failed: list = field(default_factory=list)      # (key, rc)
    empty: int = 0
    empty_cells: list = field(default_factory=list)  # (key, face) of the cells dropped as empty
    degenerate: int = 0
    seeds: list = field(default_factory=list)       # (key, point)

    def by_key(self) -> dict:
        return {f.key: f for f in self.faces}

    def vertex_key(self, f: Face, i: int):
        a, b = f.vertex_pair(i)
        k = f.key
        for p in (a, b):
            if p < self.N:
                k &= ~(1 << p)
        return (a, b, k)

    def assemble(self):
        """Vertex dedup by combinatorial key; returns (xyz (V x 3), face index lists, vkeys)."""
        index, xyz, faces = {}, [], []
        for f in self.faces:
            idx = []
            for i in range(len(f.edges)):
                vk = self.vertex_key(f, i)
                if vk not in index:
                    index[vk] = len(xyz)
                    xyz.append(f.verts[i])
                idx.append(index[vk])
            faces.append(idx)
        vkeys = [None] * len(index)
        for vk, i in index.items():
            vkeys[i] = vk
        return np.asarray(xyz).reshape(-1, 3), faces, vkeys

    def open_faces(self) -> int:
        return sum(1 for f in self.faces if any(e >= self.N for e in f.edges))


def solve_cell(net: OracleNet, key: int, start, x, box=DEFAULT_BOX, delta=DEFAULT_DELTA):
    """Face of one cell by Alg. 2 (start=None: nearest in-plane line to x)."""
    s = key_to_state(key, net.N)
    C, aF = net.cell_rows(s, box)
    if start is None:
        start = nearest_line(C, aF, x, lib=net.lib)
        if start < 0:
            return None, -1
    rc, V, pairs, nd = face_pivot(C, aF, start, x, delta, max_v=min(C.shape[0] + 1, 4096), lib=net.lib)
    if rc != 0:
        return None, rc
    return face_from_pivot(key, V, pairs, aF, nd), 0


def seed_cells(net: OracleNet, origins, dirs, R=2.0):
    seeds = []
    for o, d in zip(np.atleast_2d(origins), np.atleast_2d(dirs)):
        rc, x, s, _ = net.seed_ray(o, d, R)
        if rc == 0:
            seeds.append((state_to_key(s), x))
    return seeds


# Reading of Sec. 4.3.1 (the paper stops at a point near the surface and says nothing about
# how its cell is then taken): the walk's last point x_T lies at distance about |F|/|g| from
# the zero crossing of its cell's affine piece along the unit gradient n = g/|g|.  The segment
# from x_T - h n to x_T + h n with h = 2|F|/|g| + TRACE_PAD therefore has F of opposite signs
# at its ends while it stays inside one cell, and the dichotomy of Sec. 4.3.2 along it (o =
# x_T - h n, d = 2h n, t in [0, 1]) yields the seed cell and its exact root.
TRACE_PAD = 1e-9


def trace_bracket(x, F, g):
    """The segment (o, d) with t in [0, 1] that brackets the zero crossing near x."""
    gn = float(np.sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]))
    n = np.asarray(g, dtype=np.float64) / gn
    h = 2.0 * abs(F) / gn + TRACE_PAD
    return x - h * n, (2.0 * h) * n


def seed_sphere_trace(net: OracleNet, starts, eta=1.0, max_steps=64, eps=1e-12):
    """Sec. 4.3.1 trigger for every start point: [(key, seed point) or None] in start order."""
    out = []
    for x0 in np.atleast_2d(starts):
        rc, x, F, g, _ = net.sphere_trace(x0, eta, max_steps, eps)
        if rc != 0:
            out.append(None)
            continue
        o, d = trace_bracket(x, F, g)
        rc, xs, s, _ = net.seed_ray(o, d, 1.0)
        out.append((state_to_key(s), xs) if rc == 0 else None)
    return out


def sign_pairs(Fvals, max_pairs):
    """Reading of Sec. 4.3.2's random sampling: the r-th sample with F > 0 is paired with the
    r-th sample with F < 0, in sample order (samples with F == 0 are not used), for r below
    min(#positive, #negative, max_pairs).  Returns [(index of x-, index of x+)]."""
    pos = [i for i, f in enumerate(Fvals) if f > 0.0]
    neg = [i for i, f in enumerate(Fvals) if f < 0.0]
    return list(zip(neg, pos))[:max_pairs]


def seed_pairs(net: OracleNet, points, max_pairs):
    """Sec. 4.3.2 trigger from sampled points: pair samples of opposite sign (sign_pairs) and
    bisect each segment from x- to x+.  [(key, seed point) or None] in pair order."""
    P = np.atleast_2d(np.asarray(points, dtype=np.float64))
    Fvals = [net.F(p) for p in P]
    out = []
    for i, j in sign_pairs(Fvals, max_pairs):
        rc, xs, s, _ = net.seed_ray(P[i], P[j] - P[i], 1.0)
        out.append((state_to_key(s), xs) if rc == 0 else None)
    return out


def march(net: OracleNet, seeds, box=DEFAULT_BOX, delta=DEFAULT_DELTA, max_cells=None) -> Mesh:
    """Algorithm 1 with Alg. 2 per cell, FIFO order.  ``seeds`` = [(key, point on its face)]."""
    mesh = Mesh(net.N, box, seeds=list(seeds))
    seen = set()
    queue = deque()
    for key, x in seeds:
        if key not in seen:
            seen.add(key)
            queue.append((key, None, np.asarray(x, dtype=np.float64)))
    area_min = 1e-24 * box * box
    done = 0
    while queue:
        if max_cells is not None and done >= max_cells:
            break
        key, start, x = queue.popleft()
        done += 1
        f, rc = solve_cell(net, key, start, x, box, delta)
        if f is None:
            mesh.failed.append((key, rc))
            continue
        if f.area() <= area_min:
            mesh.empty += 1
            mesh.empty_cells.append((key, f))
            continue
        mesh.faces.append(f)
        mesh.degenerate += f.ndeg
        m = len(f.edges)
        for j, e in enumerate(f.edges):
            if e < net.N:
                nk = key ^ (1 << e)
                if nk not in seen:
                    seen.add(nk)
                    queue.append((nk, e, 0.5 * (f.verts[j] + f.verts[(j + 1) % m])))
    return mesh


def mesh_from_rays(mlp, origins, dirs, R=2.0, box=DEFAULT_BOX, delta=DEFAULT_DELTA, max_cells=None,
                   lib=None):
    net = OracleNet(mlp, lib=lib)
    seeds = seed_cells(net, origins, dirs, R)
    return net, march(net, seeds, box, delta, max_cells)
