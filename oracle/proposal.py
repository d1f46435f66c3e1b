"""FP64 CPU reference for the learned constraint proposal (test infrastructure only).

The proposal is a small MLP that, for one analytic cell, scores every hidden neuron of the
meshed net by how likely its plane carries an edge of the cell's face (the boundary planes of
Alg. 1 step 10).  The paper has no learned part; this is the plain definition the CUDA
kernels are checked against:

  features x (7 + L): entry point p (3), unit face-plane normal n = a_F[0:3] / |a_F[0:3]| (3),
                      plane offset a_F[3] / |a_F[0:3]| (1), active fraction of each hidden
                      layer (L)
  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3, score = sigmoid(z)
  loss = mean over samples and outputs of BCE(sigmoid(z), y)
       = mean(softplus(z) - y z)
Gradients by plain backpropagation; pinned by central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np


def init_params(n_in: int, hidden: int, n_out: int, seed: int = 0):
    """Kaiming-normal hidden layers, zero biases; output bias at logit(1/32) so that the
    initial scores match the sparse labels (a face has few edges among many neurons)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, np.sqrt(2.0 / n_in), (hidden, n_in))
    W2 = rng.normal(0.0, np.sqrt(2.0 / hidden), (hidden, hidden))
    W3 = rng.normal(0.0, np.sqrt(1.0 / hidden), (n_out, hidden))
    b1 = np.zeros(hidden)
    b2 = np.zeros(hidden)
    b3 = np.full(n_out, np.log(1.0 / 31.0))
    return {"W1": W1, "b1": b1, "W2": W2, "b2": b2, "W3": W3, "b3": b3}


def forward(P, X):
    """X: (B, n_in).  Returns logits (B, n_out) and the cache for backward."""
    a1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ P["W3"].T + P["b3"]
    return z, (X, a1, h1, a2, h2)


def loss(z, Y):
    """Mean binary cross-entropy with logits."""
    sp = np.logaddexp(0.0, z)
    return float(np.mean(sp - Y * z))


def backward(P, z, Y, cache):
    """Gradients of the mean BCE w.r.t. every parameter."""
    X, a1, h1, a2, h2 = cache
    B, n_out = z.shape
    dz = (1.0 / (1.0 + np.exp(-z)) - Y) / (B * n_out)
    g = {"W3": dz.T @ h2, "b3": dz.sum(0)}
    dh2 = dz @ P["W3"]
    da2 = dh2 * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    dh1 = da2 @ P["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(0)
    return g


def features(p, aF, key: int, widths):
    """Feature vector of a cell entered through point p whose face plane is aF (Eq. 12):
    p (3), aF[0:3] / |aF[0:3]| (3), aF[3] / |aF[0:3]| (1), active fraction of each layer (L)."""
    g = float(np.linalg.norm(aF[:3]))
    frac, r = [], 0
    for n in widths:
        frac.append(sum((key >> (r + i)) & 1 for i in range(n)) / n)
        r += n
    return np.concatenate([np.asarray(p, dtype=np.float64), np.asarray(aF[:3]) / g, [aF[3] / g], frac])


def face_samples(mesh, widths):
    """(features, labels, (key, edge plane) per sample) from an oracle Mesh.

    One sample per corner of every face: the entry point is the midpoint of the edge that
    leaves the corner (the point the march enters the neighbour across that edge through),
    the labels mark the neurons that carry an edge of the face (Alg. 1 step 10)."""
    N = int(sum(widths))
    X, Y, tags = [], [], []
    for f in mesh.faces:
        y = np.zeros(N)
        y[[e for e in f.edges if e < N]] = 1.0
        m = len(f.edges)
        for j in range(m):
            X.append(features(0.5 * (f.verts[j] + f.verts[(j + 1) % m]), f.aF, f.key, widths))
            Y.append(y)
            tags.append((f.key, f.edges[j]))
    return np.asarray(X).reshape(-1, 7 + len(widths)), np.asarray(Y).reshape(-1, N), tags
