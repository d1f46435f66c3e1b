"""Seeded generators for the synthetic ReLU-MLP implicit surfaces.

A network is F = f o T with hidden layers h_l = relu(W_l u_l + b_l)
(Sec. 2.2, Eq. 1; biases kept, the paper omits them only for notation) and a
linear regressor F = w_out . h_L + b_out.  The input of layer 1 is [x; z]
where z is an optional fixed latent code.  With ``skip_layer = s`` (1-based)
the input of hidden layer s is concat(h_{s-1}, [x; z]) (a DeepSDF-style
skip-concat shortcut, cf. Sec. 5.1).

Nothing in here evaluates, composes or meshes a network: these are inputs
only, shared by the CPU oracle and the CUDA path.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class MLP:
    weights: list            # W_l, float64 array (n_l, fan_in_l)
    biases: list             # b_l, float64 array (n_l,)
    w_out: np.ndarray        # (n_L,)
    b_out: float
    latent: np.ndarray | None = None   # z (latent_dim,), fixed per network
    skip_layer: int = 0      # 0 = none, else 1-based hidden layer taking concat(h_{l-1}, [x; z])
    name: str = ""
    meta: dict = field(default_factory=dict)
    slope: float = 0.0       # hidden activation a (a > 0), slope * a otherwise: 0 = ReLU, else leaky
    shortcuts: dict = field(default_factory=dict)   # residual blocks {l: (src, S or None = identity)}
    heads: list = field(default_factory=list)        # max pooling: [(w_i, b_i)], F = max_i w_i . h_L + b_i

    @property
    def widths(self) -> list:
        return [int(w.shape[0]) for w in self.weights]

    @property
    def L(self) -> int:
        return len(self.weights)

    @property
    def N(self) -> int:
        return int(sum(self.widths))

    @property
    def latent_dim(self) -> int:
        return 0 if self.latent is None else int(self.latent.shape[0])

    @property
    def in_dim(self) -> int:
        return 3 + self.latent_dim

    def fan_in(self, l: int) -> int:
        """fan-in of 1-based hidden layer l."""
        if l == 1:
            return self.in_dim
        return self.widths[l - 2] + (self.in_dim if l == self.skip_layer else 0)

    def validate(self) -> None:
        assert self.L >= 1
        assert self.skip_layer == 0 or 2 <= self.skip_layer <= self.L
        for l in range(1, self.L + 1):
            W, b = self.weights[l - 1], self.biases[l - 1]
            assert W.dtype == np.float64 and b.dtype == np.float64
            assert W.shape == (self.widths[l - 1], self.fan_in(l)), (l, W.shape)
            assert b.shape == (self.widths[l - 1],)
        assert self.w_out.shape == (self.widths[-1],)
        for w, b in self.heads:
            assert w.shape == (self.widths[-1],) and np.isscalar(b)
        assert len(self.heads) != 1
        for l, (src, S) in self.shortcuts.items():
            assert 1 <= l <= self.L and 0 <= src < l, (l, src)
            n_s = 3 if src == 0 else self.widths[src - 1]
            if S is None:
                assert n_s == self.widths[l - 1], (l, src)
            else:
                assert S.shape == (self.widths[l - 1], n_s), (l, S.shape)


# --------------------------------------------------------------------------------------------
# hand-built closed-form surfaces


def octahedron(C: float = 10.0) -> MLP:
    """F(x) = |x|_1 - 1 as a 3 -> 6 -> 1 ReLU net.

    |t| = 2 relu(t) - t and t = relu(t + C) - C for t > -C, so
    F = sum_i [2 relu(x_i) - relu(x_i + C)] + 3C - 1.  Exact mesh: the regular
    octahedron with vertices +-e_i, one triangle per orthant.
    """
    W1 = np.zeros((6, 3))
    b1 = np.zeros(6)
    for i in range(3):
        W1[i, i] = 1.0
        W1[3 + i, i] = 1.0
        b1[3 + i] = C
    w_out = np.array([2.0, 2.0, 2.0, -1.0, -1.0, -1.0])
    m = MLP([W1], [b1], w_out, 3 * C - 1.0, name="octahedron")
    m.validate()
    return m


def fibonacci_normals(n: int = 12, seed: int = 1, jitter: float = 1e-3) -> np.ndarray:
    """n unit normals on a Fibonacci sphere, each jittered by N(0, jitter^2) and renormalised."""
    rng = np.random.default_rng(seed)
    i = np.arange(n) + 0.5
    phi = np.arccos(1.0 - 2.0 * i / n)
    theta = np.pi * (1.0 + 5.0 ** 0.5) * i
    P = np.stack([np.cos(theta) * np.sin(phi), np.sin(theta) * np.sin(phi), np.cos(phi)], 1)
    P = P + rng.normal(0.0, jitter, P.shape)
    return P / np.linalg.norm(P, axis=1, keepdims=True)


def polytope_max_of_planes(seed: int = 1, offset: float = 0.5, C: float = 10.0) -> MLP:
    """F(x) = max_i (n_i . x - offset) over 12 planes as a 3->12->6->3->2->1 ReLU net.

    Pairwise max(a, b) = relu(a - b) + relu(b + C) - C (valid while b > -C),
    arranged as a tree: 12 planes -> 6 maxes -> 3 -> (max of 2, carry 1) -> 1.
    The zero set is the boundary of the convex polytope {n_i . x <= offset}.
    """
    Nn = fibonacci_normals(12, seed)
    p_w, p_b = Nn, -offset * np.ones(12)
    # layer 1: for pair j: relu(p_{2j} - p_{2j+1}), relu(p_{2j+1} + C)
    W1 = np.zeros((12, 3)); b1 = np.zeros(12)
    for j in range(6):
        a, b = 2 * j, 2 * j + 1
        W1[2 * j] = p_w[a] - p_w[b]; b1[2 * j] = p_b[a] - p_b[b]
        W1[2 * j + 1] = p_w[b]; b1[2 * j + 1] = p_b[b] + C
    # m_j = h1[2j] + h1[2j+1] - C ; layer 2: pairs (m_{2i}, m_{2i+1})
    W2 = np.zeros((6, 12)); b2 = np.zeros(6)
    for i in range(3):
        W2[2 * i, 4 * i: 4 * i + 2] = 1.0; W2[2 * i, 4 * i + 2: 4 * i + 4] = -1.0
        W2[2 * i + 1, 4 * i + 2: 4 * i + 4] = 1.0
    # q_i = h2[2i] + h2[2i+1] - C ; layer 3: relu(q0 - q1), relu(q1 + C), relu(q2 + C)
    W3 = np.zeros((3, 6)); b3 = np.zeros(3)
    W3[0, 0:2] = 1.0; W3[0, 2:4] = -1.0
    W3[1, 2:4] = 1.0
    W3[2, 4:6] = 1.0
    # r = h3[0] + h3[1] - C, q2 = h3[2] - C ; layer 4: relu(r - q2), relu(q2 + C)
    W4 = np.zeros((2, 3)); b4 = np.zeros(2)
    W4[0, 0:2] = 1.0; W4[0, 2] = -1.0
    W4[1, 2] = 1.0
    m = MLP([W1, W2, W3, W4], [b1, b2, b3, b4], np.array([1.0, 1.0]), -C,
            name="polytope12", meta={"normals": Nn, "offset": offset})
    m.validate()
    return m


# --------------------------------------------------------------------------------------------
# geometric-init networks


def _value_at_origin(m: MLP) -> float:
    """F(0) of the network (plain numpy evaluation of Eq. 1, with its shortcuts and slope)."""
    u0 = np.zeros(3) if m.latent is None else np.concatenate([np.zeros(3), m.latent])
    hs = [np.zeros(3)]
    for l, (W, b) in enumerate(zip(m.weights, m.biases), start=1):
        inp = u0 if l == 1 else (np.concatenate([hs[-1], u0]) if l == m.skip_layer else hs[-1])
        a = W @ inp + b
        if l in m.shortcuts:
            src, S = m.shortcuts[l]
            a = a + (hs[src] if S is None else S @ hs[src])
        hs.append(np.where(a > 0.0, a, m.slope * a))
    return float(m.w_out @ hs[-1] + m.b_out)


def geometric_init(widths, seed: int, sigma: float, radius: float = 0.6,
                   latent_dim: int = 0, latent_std: float = 0.0, skip_layer: int = 0,
                   name: str = "", recenter: bool = False) -> MLP:
    """Geometric sphere initialisation, then every parameter perturbed by N(0, sigma^2).

    Hidden W ~ N(0, 2 / n_out), b = 0; output w ~ N(sqrt(pi)/sqrt(n_L), 1e-6^2),
    b_out = -radius, which makes F(x) ~ |x| - radius before the perturbation
    (geometric initialisation of Atzmon & Lipman, SAL, 2020).  The skip layer's
    weights are scaled by 1/sqrt(2) so that the concatenated input keeps the
    norm of a plain layer's input.

    recenter: shift b_out after the perturbation so that F(0) = -radius again.  In deep,
    wide nets the rectified bias perturbations add up to a positive offset (F ~ 3 over the
    whole box for 3-[256]x8-1 at sigma = 0.05) that leaves no zero level set; the shift
    restores the surface around the origin.
    """
    rng = np.random.default_rng(seed)
    widths = [int(w) for w in widths]
    in_dim = 3 + latent_dim
    latent = rng.normal(0.0, latent_std, latent_dim) if latent_dim else None
    Ws, bs = [], []
    for l, n in enumerate(widths, start=1):
        fan = in_dim if l == 1 else widths[l - 2] + (in_dim if l == skip_layer else 0)
        W = rng.normal(0.0, np.sqrt(2.0 / n), (n, fan))
        if l == skip_layer:
            W /= np.sqrt(2.0)
        Ws.append(W)
        bs.append(np.zeros(n))
    nL = widths[-1]
    w_out = rng.normal(np.sqrt(np.pi) / np.sqrt(nL), 1e-6, nL)
    b_out = -radius
    if sigma > 0:
        Ws = [W + rng.normal(0.0, sigma, W.shape) for W in Ws]
        bs = [b + rng.normal(0.0, sigma, b.shape) for b in bs]
        w_out = w_out + rng.normal(0.0, sigma, w_out.shape)
        b_out = b_out + float(rng.normal(0.0, sigma))
    m = MLP(Ws, bs, w_out, float(b_out), latent=latent, skip_layer=skip_layer, name=name,
            meta={"seed": seed, "sigma": sigma, "radius": radius, "recentered": recenter})
    if recenter:
        m.b_out = float(m.b_out - (_value_at_origin(m) + radius))
    m.validate()
    return m


def residual_net(seed: int = 31, width: int = 24, depth: int = 5, sigma: float = 0.05, radius: float = 0.6,
                 v_scale: float = 0.1, t_scale: float = 0.25) -> MLP:
    """3 -> [width] x depth -> 1 with the residual blocks of Sec. 5.1: a block of the second kind
    (g(V x + T x), V ~ v_scale N(0, 1), width x 3) ending at layer 2, and blocks of the first kind
    (g(h + T h), the identity from the layer before the block) over layers 3-4, 5-6, ...  The
    branch T of a first-kind block is a geometric-init layer pair scaled by t_scale, so each
    block stays close to the identity and the net close to a sphere's distance function; F(0)
    is recentred to -radius."""
    m = geometric_init([width] * depth, seed, sigma, radius=radius, name=f"residual_w{width}_d{depth}_s{seed}")
    rng = np.random.default_rng(seed + 1000)
    sc = {2: (0, v_scale * rng.normal(size=(width, 3)))}
    for q in range(4, depth + 1, 2):
        sc[q] = (q - 2, None)
        m.weights[q - 2] = t_scale * m.weights[q - 2]
        m.weights[q - 1] = t_scale * m.weights[q - 1]
    m.shortcuts = sc
    m.b_out = float(m.b_out - (_value_at_origin(m) + radius))
    m.meta["shortcuts"] = {int(k): int(v[0]) for k, v in sc.items()}
    m.validate()
    return m


def pooled_net(seed: int = 61, count: int = 4, width: int = 32, depth: int = 4, sigma: float = 0.05,
               radius: float = 0.6, offset: float = 0.2) -> MLP:
    """Sec. 5.2's final max pooling over `count` sub-networks 3 -> [width] x depth -> 1 (the shape
    of the paper's local decoder, 4 x D4-W32): sub-network i is a geometric-init sphere net
    (seed + i, recentred) moved to the centre c_i = offset e_i (e_i = +x, -x, +y, -y, +z, -z, ...),
    and F = max_i F_i, whose negative side is the intersection of theirs.  Returned as one MLP
    whose hidden layers hold the sub-networks side by side (block-diagonal weights, the units of
    sub-network i at i * width of every layer) and whose `heads` are [(w_i, b_i)], head i reading
    sub-network i's last-layer units only.  meta["subnet_width"] = width."""
    dirs = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
    subs = []
    for i in range(count):
        g = geometric_init([width] * depth, seed + i, sigma, radius=radius, recenter=True)
        c = offset * dirs[i % 6] * (1 + i // 6)
        g.biases[0] = g.biases[0] - g.weights[0] @ c          # F_i(x) = G_i(x - c_i)
        subs.append(g)
    n = count * width
    Ws, bs = [], []
    for l in range(depth):
        if l == 0:
            W = np.vstack([g.weights[0] for g in subs])
        else:
            W = np.zeros((n, n))
            for i, g in enumerate(subs):
                W[i * width:(i + 1) * width, i * width:(i + 1) * width] = g.weights[l]
        Ws.append(W)
        bs.append(np.concatenate([g.biases[l] for g in subs]))
    heads = []
    for i, g in enumerate(subs):
        w = np.zeros(n)
        w[i * width:(i + 1) * width] = g.w_out
        heads.append((w, float(g.b_out)))
    m = MLP(Ws, bs, heads[0][0].copy(), heads[0][1], name=f"pooled{count}_w{width}_d{depth}_s{seed}",
            meta={"seed": seed, "sigma": sigma, "subnet_width": width, "count": count}, heads=heads)
    m.validate()
    return m


def sphere_net(seed: int = 2, width: int = 64, depth: int = 4, sigma: float = 0.05) -> MLP:
    """3 -> [width] x depth -> 1, geometric init + N(0, sigma^2) bumps (the 3-[64]x4-1 workload)."""
    return geometric_init([width] * depth, seed, sigma, name=f"sphere_w{width}_d{depth}_s{seed}")


def decoder_net(seed: int = 3, width: int = 512, depth: int = 8, latent_dim: int = 256,
                skip_layer: int = 4, sigma: float = 0.02) -> MLP:
    """(3 + latent) -> [width] x depth -> 1 with skip-concat of [x; z] at hidden layer 4."""
    return geometric_init([width] * depth, seed, sigma, latent_dim=latent_dim, latent_std=0.01,
                          skip_layer=skip_layer, name=f"decoder_w{width}_d{depth}_s{seed}", recenter=True)


def batch_nets(master_seed: int = 4, count: int = 64) -> list:
    """count independent nets 3 -> [w] x d -> 1, w in {32,64,128,256}, d in {4,6,8}, sigma ~ U[0.02, 0.1]."""
    rng = np.random.default_rng(master_seed)
    out = []
    for i in range(count):
        w = int(rng.choice([32, 64, 128, 256]))
        d = int(rng.choice([4, 6, 8]))
        s = float(rng.uniform(0.02, 0.1))
        sub = int(rng.integers(0, 2 ** 31 - 1))
        out.append(geometric_init([w] * d, sub, s, name=f"batch{i}_w{w}_d{d}", recenter=True))
    return out


def proposal_target_net(seed: int = 5, width: int = 256, depth: int = 8, sigma: float = 0.05) -> MLP:
    return geometric_init([width] * depth, seed, sigma, name=f"proposal_w{width}_d{depth}_s{seed}", recenter=True)


def proposal_train_nets(seeds=range(100, 132), width: int = 256, depth: int = 8, sigma: float = 0.05) -> list:
    """The learned proposal's training nets: independent nets of the target net's shape and
    recipe (3 -> [256] x 8 -> 1, geometric init, sigma 0.05, recentred) with seeds 100-131; the
    target net (seed 5) is not among them."""
    return [proposal_target_net(seed=int(s), width=width, depth=depth, sigma=sigma) for s in seeds]


def sibling(mlp: MLP, seed: int, sigma: float = 0.005) -> MLP:
    """The same network with every hidden weight and bias moved by N(0, sigma^2): a nearby
    checkpoint of it (the training nets of the learned proposal)."""
    rng = np.random.default_rng(seed)
    m = MLP([w + rng.normal(0.0, sigma, w.shape) for w in mlp.weights],
            [b + rng.normal(0.0, sigma, b.shape) for b in mlp.biases],
            mlp.w_out.copy(), float(mlp.b_out), None if mlp.latent is None else mlp.latent.copy(),
            mlp.skip_layer, f"{mlp.name}_sib{seed}", dict(mlp.meta), mlp.slope, dict(mlp.shortcuts))
    m.validate()
    return m


def leaky(mlp: MLP, slope: float) -> MLP:
    """The same network with the leaky / parametric ReLU g(a) = a (a > 0), slope * a (a <= 0)."""
    import copy
    m = copy.deepcopy(mlp)
    m.slope = float(slope)
    m.name = f"{mlp.name}_leaky{slope:g}"
    return m


def tiny_net(widths, seed: int, sigma: float = 0.1, radius: float = 0.6) -> MLP:
    """Small geometric-init nets (<= 16 ReLUs) for exhaustive enumeration."""
    return geometric_init(list(widths), seed, sigma, radius=radius,
                          name=f"tiny_{'x'.join(map(str, widths))}_s{seed}")


# --------------------------------------------------------------------------------------------
# seed rays


def seed_rays(n: int = 1, seed: int = 0, length: float = 2.0, direction=None):
    """Rays (origin, unit direction, length) from the origin.

    n = 1 with no direction gives the single +x ray; otherwise directions are
    drawn uniformly on the sphere from ``seed``.
    """
    if direction is not None:
        d = np.asarray(direction, dtype=np.float64).reshape(1, 3)
        d = d / np.linalg.norm(d)
        d = np.repeat(d, n, 0)
    elif n == 1:
        d = np.array([[1.0, 0.0, 0.0]])
    else:
        rng = np.random.default_rng(seed)
        d = rng.normal(size=(n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.zeros((n, 3))
    return o, d, float(length)


def trigger_points(n: int, seed: int = 0, box: float = 1.5) -> np.ndarray:
    """n points drawn uniformly from the cube [-box, box]^3: start points for the
    sphere-tracing trigger and samples for the random-pair trigger."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-box, box, size=(n, 3))
