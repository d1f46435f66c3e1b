"""Independent references used to pin the oracle.

Each helper here computes a quantity of the method by a route that shares
nothing with the oracle's code: the network's pre-activations by torch's
``nn.functional.linear`` (a library routine), a region's affine maps by
evaluating the masked network at four points (the definition of an affine
map), cell and face feasibility by linear programs (scipy's HiGHS), face
polygons by scipy's ``HalfspaceIntersection`` (Qhull), and the max-of-planes
polytope by ``ConvexHull``.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------------------------
# forward pass by torch (library routine)


def torch_forward(mlp, X):
    """Pre-activations (P, N) and F (P,) of the MLP at points X (P, 3), FP64 torch CPU."""
    import torch
    import torch.nn.functional as tf

    X = torch.as_tensor(np.atleast_2d(X), dtype=torch.float64)
    if mlp.latent is not None:
        z = torch.as_tensor(mlp.latent, dtype=torch.float64).expand(X.shape[0], -1)
        u0 = torch.cat([X, z], 1)
    else:
        u0 = X
    h, pres = None, []
    for l, (W, b) in enumerate(zip(mlp.weights, mlp.biases), start=1):
        inp = u0 if l == 1 else (torch.cat([h, u0], 1) if l == mlp.skip_layer else h)
        a = tf.linear(inp, torch.as_tensor(W), torch.as_tensor(b))
        pres.append(a)
        h = torch.relu(a)
    F = tf.linear(h, torch.as_tensor(mlp.w_out)[None, :], torch.as_tensor([mlp.b_out], dtype=torch.float64))
    return torch.cat(pres, 1).numpy(), F[:, 0].numpy()


# --------------------------------------------------------------------------------------------
# affine maps of a region by evaluating the masked network at 0, e_x, e_y, e_z


def masked_eval(mlp, s, X):
    """Pre-activations and F with every hidden state frozen to the pattern s (no ReLU)."""
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    u0 = X if mlp.latent is None else np.hstack([X, np.broadcast_to(mlp.latent, (X.shape[0], mlp.latent_dim))])
    h, pres, off = None, [], 0
    for l, (W, b) in enumerate(zip(mlp.weights, mlp.biases), start=1):
        inp = u0 if l == 1 else (np.hstack([h, u0]) if l == mlp.skip_layer else h)
        a = inp @ W.T + b
        pres.append(a)
        n = W.shape[0]
        h = a * s[off: off + n][None, :]
        off += n
    F = h @ mlp.w_out + mlp.b_out
    return np.hstack(pres), F


def masked_affine_maps(mlp, s):
    """Rows [c | c0] of every neuron and of F for the frozen pattern s: c0 = value at 0,
    c_i = value at e_i minus value at 0."""
    P = np.vstack([np.zeros(3), np.eye(3)])
    pre, F = masked_eval(mlp, np.asarray(s, dtype=np.float64), P)
    A = np.zeros((pre.shape[1], 4))
    A[:, 3] = pre[0]
    A[:, :3] = (pre[1:] - pre[0]).T
    aF = np.array([F[1] - F[0], F[2] - F[0], F[3] - F[0], F[0]])
    return A, aF


# --------------------------------------------------------------------------------------------
# linear programs (HiGHS)


def chebyshev_lp(rows, box, plane=None, plane_frame=None):
    """max t s.t. r_k . [x;1] + t * w_k <= 0 for every row, |x_i| + t <= box, t <= 1
    (and a_F . [x;1] = 0 when ``plane`` is given).  w_k is the row's normal norm, measured
    in the plane when a plane is given.  Returns (t*, x*) or (-inf, None)."""
    from scipy.optimize import linprog

    rows = np.asarray(rows, dtype=np.float64)
    if plane is not None:
        n = plane[:3] / np.linalg.norm(plane[:3])
        proj = rows[:, :3] - np.outer(rows[:, :3] @ n, n)
        w = np.linalg.norm(proj, axis=1)
    else:
        w = np.linalg.norm(rows[:, :3], axis=1)
    A_ub = [np.hstack([rows[:, :3], w[:, None]])]
    b_ub = [-rows[:, 3]]
    for i in range(3):
        for sg in (1.0, -1.0):
            r = np.zeros(4); r[i] = sg; r[3] = 1.0
            A_ub.append(r[None, :]); b_ub.append(np.array([box]))
    A_ub = np.vstack(A_ub); b_ub = np.concatenate(b_ub)
    kw = {}
    if plane is not None:
        kw["A_eq"] = np.array([[plane[0], plane[1], plane[2], 0.0]])
        kw["b_eq"] = np.array([-plane[3]])
    res = linprog(c=[0, 0, 0, -1.0], A_ub=A_ub, b_ub=b_ub, bounds=[(None, None)] * 3 + [(None, 1.0)],
                  method="highs", **kw)
    if res.status != 0:
        return -np.inf, None
    return -res.fun, res.x[:3]


def enumerate_faces(mlp, box, eps=1e-9):
    """Exhaustive search over all 2^N activation patterns of a small net (N <= 16).

    Patterns are grown neuron by neuron in layer order; a prefix is dropped only when its
    cell (the rows of its neurons, which depend on earlier states only) has no interior in
    the box, which no completion can repair.  For every full pattern whose cell has an
    interior, the face LP decides whether a_F . x = 0 meets the cell in a 2-D region.
    Returns {key: interior point of the face}.
    """
    N = mlp.N
    faces = {}
    tol_cells = [0]

    def rows_for(s_prefix, k):
        # rows of the first k neurons for the prefix; the state of neurons >= k does not
        # influence them (they only depend on earlier layers)
        s = np.zeros(N)
        s[:len(s_prefix)] = s_prefix
        A, _ = masked_affine_maps(mlp, s)
        sg = 1.0 - 2.0 * s[:k]
        return A[:k] * sg[:, None]

    def rec(prefix):
        k = len(prefix)
        if k == N:
            s = np.array(prefix, dtype=np.float64)
            A, aF = masked_affine_maps(mlp, s)
            C = A * (1.0 - 2.0 * s)[:, None]
            if np.linalg.norm(aF[:3]) == 0:
                return
            t, x = chebyshev_lp(C, box, plane=aF)
            if t > eps:
                key = int(sum(int(b) << i for i, b in enumerate(prefix)))
                faces[key] = x
            return
        for b in (0, 1):
            p = prefix + [b]
            C = rows_for(p, k + 1)
            zero = np.linalg.norm(C[:, :3], axis=1) == 0
            if np.any(C[zero, 3] > 0):
                continue
            t, _ = chebyshev_lp(C[~zero], box)
            tol_cells[0] += 1
            if t > eps:
                rec(p)

    rec([])
    return faces


# --------------------------------------------------------------------------------------------
# polygons by Qhull


def halfspace_polygon(C, aF, interior, box):
    """Vertices of {a_F . x = 0, C [x;1] <= 0} (C may already hold box rows) by scipy's
    HalfspaceIntersection in a 2-D frame of the face plane; returned in 3-D, unordered."""
    from scipy.spatial import HalfspaceIntersection

    n = aF[:3] / np.linalg.norm(aF[:3])
    p0 = -aF[3] * aF[:3] / (aF[:3] @ aF[:3])
    u = np.cross(n, [1.0, 0.0, 0.0])
    if np.linalg.norm(u) < 0.5:
        u = np.cross(n, [0.0, 1.0, 0.0])
    u /= np.linalg.norm(u)
    w = np.cross(n, u)
    hs = []
    for r in C:
        a, b, g = r[:3] @ u, r[:3] @ w, r[:3] @ p0 + r[3]
        if a == 0 and b == 0:
            continue
        hs.append([a, b, g])
    ip = np.array([(interior - p0) @ u, (interior - p0) @ w])
    hsi = HalfspaceIntersection(np.array(hs), ip)
    P = hsi.intersections
    return p0[None, :] + P[:, :1] * u[None, :] + P[:, 1:2] * w[None, :]


def polytope_facets(normals, offset):
    """Convex polytope {n_i . x <= offset}: per-plane facet area, volume and vertices."""
    from scipy.spatial import ConvexHull, HalfspaceIntersection

    hs = np.hstack([normals, -offset * np.ones((len(normals), 1))])
    V = HalfspaceIntersection(hs, np.zeros(3)).intersections
    hull = ConvexHull(V)
    area = np.zeros(len(normals))
    for simplex, eq in zip(hull.simplices, hull.equations):
        i = int(np.argmin(np.abs(normals @ eq[:3] - 1.0) + np.abs(-eq[3] - offset)))
        a, b, c = V[simplex]
        area[i] += 0.5 * np.linalg.norm(np.cross(b - a, c - a))
    return area, hull.volume, V


# --------------------------------------------------------------------------------------------
# mesh invariants


def mesh_edges(faces_idx):
    E = {}
    for fi, f in enumerate(faces_idx):
        m = len(f)
        for i in range(m):
            e = (min(f[i], f[(i + 1) % m]), max(f[i], f[(i + 1) % m]))
            E.setdefault(e, []).append(fi)
    return E


def euler_characteristic(n_vertices, faces_idx):
    return n_vertices - len(mesh_edges(faces_idx)) + len(faces_idx)


def signed_volume(xyz, faces_idx):
    vol = 0.0
    for f in faces_idx:
        a = xyz[f[0]]
        for i in range(1, len(f) - 1):
            vol += np.dot(a, np.cross(xyz[f[i]], xyz[f[i + 1]])) / 6.0
    return vol
