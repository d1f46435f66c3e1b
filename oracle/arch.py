"""Oracle for the architectures of Sec. 5: MLPs with residual blocks (Sec. 5.1) and a final
max pooling over sub-networks (Sec. 5.2).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: plain FP64 numpy loops for the
network algebra, the oracle's own Alg. 2 (``am_oracle.c`` through ``oracle.face_pivot``) for
each face, and a literal FIFO rendering of Alg. 1 for the march.

Residual network (``ResNet``).  h_0 = x (3-d input) and, for the hidden layers l = 1..L,
    a_l = W_l h_{l-1} + b_l + S_l h_{src(l)},    h_l = ReLU(a_l),    F = w_out . h_L + b_out.
A residual block over the layers p..q has its shortcut on its last layer: src(q) = p - 1, and
S_q = I for the first kind of block (g(x + T_PreAct x), which needs n_{p-1} = n_q) or a
matrix V for the second kind (g(V x + T_PreAct x)).  Layers without a shortcut are plain.
Within a cell of state pattern s (Def. 2, a tie giving 0) every pre-activation is affine in x:
    Z_0 = [I | 0],  Z_l = W_l H_{l-1} + [0 | b_l] + S_l H_{src(l)},  H_l = diag(s_l) Z_l,
    a_F = w_out H_L + [0 | b_out],
which is the region-wise mapping of a residual block (Sec. 5.1: diag(s_L)(I + W_L prod W_l^r)
for the first kind) chained through the network; the rows of Z_l are the neuron-wise maps.

Max pooling (``MaxPool``).  F = max_i F_(i) over M sub-networks that share the input.  A cell
is the pattern of every sub-network's units (concatenated, N = sum N_(i) bits) together with
the index j of the pooled maximum (the state functional e_j of Sec. 5.2; on a tie the smallest
index).  Its system is the sign-adjusted unit rows of every sub-network and, for every i != j,
the row a_F(i) - a_F(j) (<= 0 in the subcell); its face lies on a_F(j).  Crossing a unit's
plane flips that unit; crossing the row of i moves the maximum to i.

Plane ids: unit k -> k (0..N-1); the pooling row of sub-network i -> N + i; the box faces
+x, -x, +y, -y, +z, -z -> N + M + 0..5.  Cell key: the unit pattern as an integer plus
j << N.  A plain ResNet is a MaxPool of one sub-network (no pooling rows, j = 0).

Leaky / parametric ReLU (the paper's closing remarks name them as the next activations): with
g(a) = a for a > 0 and slope * a otherwise, the state functional and hence the cells are those
of Def. 2 unchanged; inside a cell the inactive units pass slope * a instead of 0, so
diag(s_l) above becomes diag(s_l + slope (1 - s_l)).
"""
from __future__ import annotations

from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import oracle as O


@dataclass
class ResNet:
    weights: list                    # W_l: n_l x n_{l-1} (n_0 = 3)
    biases: list                     # b_l: n_l
    w_out: np.ndarray                # n_L
    b_out: float
    shortcuts: dict = field(default_factory=dict)   # q -> (src, S or None for the identity)
    slope: float = 0.0               # leaky / parametric ReLU: g(a) = a (a > 0), slope * a (a <= 0)

    @property
    def widths(self):
        return [W.shape[0] for W in self.weights]

    @property
    def N(self) -> int:
        return int(sum(self.widths))


def res_forward(net: ResNet, x):
    """Pre-activations of every unit (layer order) and F at the point x."""
    hs = [np.asarray(x, dtype=np.float64)]
    pre = []
    for l, (W, b) in enumerate(zip(net.weights, net.biases), start=1):
        a = W @ hs[l - 1] + b
        if l in net.shortcuts:
            src, S = net.shortcuts[l]
            a = a + (hs[src] if S is None else S @ hs[src])
        pre.append(a)
        hs.append(np.where(a > 0.0, a, net.slope * a))
    return np.concatenate(pre), float(net.w_out @ hs[-1] + net.b_out)


def res_compose(net: ResNet, s):
    """Neuron-wise affine maps (N x 4, layer order) and a_F (4,) of the cell with pattern s."""
    s = np.asarray(s)
    Hs = [np.hstack([np.eye(3), np.zeros((3, 1))])]
    rows, off = [], 0
    for l, (W, b) in enumerate(zip(net.weights, net.biases), start=1):
        n = W.shape[0]
        Z = W @ Hs[l - 1]
        Z[:, 3] += b
        if l in net.shortcuts:
            src, S = net.shortcuts[l]
            Z = Z + (Hs[src] if S is None else S @ Hs[src])
        rows.append(Z)
        g = np.where(s[off:off + n] > 0, 1.0, net.slope)          # diag of the cell's slopes
        Hs.append(Z * g[:, None])
        off += n
    aF = net.w_out @ Hs[-1]
    aF[3] += net.b_out
    return np.vstack(rows), aF


@dataclass
class MaxPool:
    subnets: list                    # ResNet each

    @property
    def M(self) -> int:
        return len(self.subnets)

    @property
    def N(self) -> int:
        return int(sum(n.N for n in self.subnets))

    def key(self, s, j) -> int:
        return O.state_to_key(np.asarray(s, dtype=np.uint8)) | (int(j) << self.N)

    def split(self, key: int):
        mask = (1 << self.N) - 1
        return O.key_to_state(key & mask, self.N), key >> self.N

    def forward(self, x):
        """(pre-activations of all units, F_(i) for every i, F, j)."""
        pres, Fs = [], []
        for n in self.subnets:
            p, f = res_forward(n, x)
            pres.append(p)
            Fs.append(f)
        j = int(np.argmax(Fs))           # first maximal index
        return np.concatenate(pres), np.asarray(Fs), float(Fs[j]), j

    def state(self, x):
        pre, _, F, j = self.forward(x)
        return (pre > 0.0).astype(np.uint8), j, F

    def cell_rows(self, s, j, box=O.DEFAULT_BOX):
        """Rows of the subcell (unit rows, pooling rows i != j, box rows), their plane ids, a_F(j)."""
        rows, aFs, off = [], [], 0
        for n in self.subnets:
            A, aF = res_compose(n, s[off:off + n.N])
            rows.append(A * (1.0 - 2.0 * np.asarray(s[off:off + n.N], dtype=np.float64))[:, None])
            aFs.append(aF)
            off += n.N
        ids = list(range(self.N))
        for i in range(self.M):
            if i != j:
                rows.append((aFs[i] - aFs[j])[None, :])
                ids.append(self.N + i)
        bx = np.zeros((6, 4))
        for k in range(3):
            bx[2 * k, k], bx[2 * k, 3] = 1.0, -box
            bx[2 * k + 1, k], bx[2 * k + 1, 3] = -1.0, -box
        rows.append(bx)
        ids += [self.N + self.M + k for k in range(6)]
        return np.vstack(rows), ids, aFs[j]

    def neighbour(self, key: int, plane: int):
        """Cell across `plane` from the cell `key`, None for a box face."""
        if plane < self.N:
            return key ^ (1 << plane)
        if plane < self.N + self.M:
            return (key & ((1 << self.N) - 1)) | ((plane - self.N) << self.N)
        return None


def as_pool(net) -> MaxPool:
    return net if isinstance(net, MaxPool) else MaxPool([net])


def seed_ray(pool: MaxPool, o, d, R=2.0, max_halvings=200):
    """Sec. 4.3.2 on the pooled F: bisect until both bracket ends are in one subcell (same
    pattern, same j), then the exact root of the affine a_F(j) on the segment."""
    o, d = np.asarray(o, dtype=np.float64), np.asarray(d, dtype=np.float64)
    slo, jlo, flo = pool.state(o)
    shi, jhi, fhi = pool.state(o + R * d)
    if not ((flo < 0.0 < fhi) or (fhi < 0.0 < flo)):
        return None
    tlo, thi = 0.0, R
    for _ in range(max_halvings):
        if jlo == jhi and np.array_equal(slo, shi):
            t = tlo + flo / (flo - fhi) * (thi - tlo)
            return pool.key(slo, jlo), o + t * d
        tm = 0.5 * (tlo + thi)
        sm, jm, fm = pool.state(o + tm * d)
        if (fm < 0.0) == (flo < 0.0) and fm != 0.0:
            tlo, slo, jlo, flo = tm, sm, jm, fm
        else:
            thi, shi, jhi, fhi = tm, sm, jm, fm
    return None


def solve_cell(pool: MaxPool, key: int, start, x, box=O.DEFAULT_BOX, delta=O.DEFAULT_DELTA):
    """Face of one subcell by Alg. 2 (start: plane id of the entry plane, None: nearest line)."""
    s, j = pool.split(key)
    C, ids, aF = pool.cell_rows(s, j, box)
    if start is None:
        r0 = O.nearest_line(C, aF, x)
        if r0 < 0:
            return None, -1
    else:
        r0 = ids.index(start)
    rc, V, pairs, nd = O.face_pivot(C, aF, r0, x, delta, max_v=min(C.shape[0] + 1, 4096))
    if rc != 0:
        return None, rc
    mapped = np.array([[ids[a], ids[b]] for a, b in pairs], dtype=np.int64)
    return O.face_from_pivot(key, V, mapped, aF, nd), 0


def march(pool: MaxPool, seeds, box=O.DEFAULT_BOX, delta=O.DEFAULT_DELTA, max_cells=None) -> O.Mesh:
    """Alg. 1 over subcells, FIFO order, from seeds = [(key, point on its face)]."""
    mesh = O.Mesh(pool.N, box, seeds=list(seeds))
    seen, queue = set(), deque()
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
        f, rc = solve_cell(pool, key, start, x, box, delta)
        if f is None:
            mesh.failed.append((key, rc))
            continue
        if f.area() <= area_min:
            mesh.empty += 1
            continue
        mesh.faces.append(f)
        mesh.degenerate += f.ndeg
        m = len(f.edges)
        for i, e in enumerate(f.edges):
            nk = pool.neighbour(key, e)
            if nk is not None and nk not in seen:
                seen.add(nk)
                queue.append((nk, e if e < pool.N else pool.N + (key >> pool.N),
                              0.5 * (f.verts[i] + f.verts[(i + 1) % m])))
    return mesh
