"""Whole-mesh checks at full size, vectorised (numpy), for meshes of millions of faces.

Test infrastructure only.  A face is named by a 128-bit fingerprint of its cell key (two
independent 64-bit hashes, each a sum over the key's 64-bit words of a mixed word), so that
the key of the neighbour across neuron plane p (the key with bit p flipped, Alg. 1 step 10)
has a fingerprint computable from the face's own in O(1): only word p // 64 changes.  With
that:

* closure: every edge on a neuron plane p has its reciprocal, i.e. the face of cell key ^ e_p
  exists and lists plane p among its edges (Thm. 1: a face's edges are shared with exactly one
  neighbouring face); every such edge is seen exactly twice;
* Euler characteristic V - E + F with E = corners / 2 on a closed surface;
* the vertex indices are one per combinatorial vertex key (lo, hi, key with bits lo and hi
  cleared), both ways;
* order-independent digests of the face set and of the edge cycles, for comparing two meshes
  (or a mesh with a stored digest of the oracle's) without holding both in memory.

The hashes hold none of the method's arithmetic; they only name keys and cycles.
"""
from __future__ import annotations

import numpy as np

_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_G = np.uint64(0x9E3779B97F4A7C15)


def mix64(x):
    """splitmix64's output function (Steele, Lea & Flood 2014) on uint64 arrays (wrapping)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _G
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _salts(kw: int, which: int) -> np.ndarray:
    return mix64(np.arange(kw, dtype=np.uint64) * np.uint64(2) + np.uint64(0x5EED0 + 7919 * which))


def _wmix(words, w, which):
    """mix of word values `words` sitting at word index w (arrays of equal length)."""
    s = _salts(int(np.max(w)) + 1 if np.size(w) else 1, which)
    return mix64(np.asarray(words, dtype=np.uint64) ^ s[w])


def face_hash(keys: np.ndarray, which: int = 0) -> np.ndarray:
    """64-bit hash of each key row (F, kw) uint64: sum over words of mix(word ^ salt_w)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    F, kw = keys.shape
    s = _salts(kw, which)
    h = np.zeros(F, dtype=np.uint64)
    with np.errstate(over="ignore"):
        for w in range(kw):
            h += mix64(keys[:, w] ^ s[w])
    return h


def _flip_hash(h, keys, f, p, which):
    """hash of key[f] with bit p flipped, from the face hash h[f] (arrays over edge instances)."""
    w = (p >> 6).astype(np.int64)
    word = keys[f, w]
    flipped = word ^ (np.uint64(1) << (p & 63).astype(np.uint64))
    with np.errstate(over="ignore"):
        return h[f] - _wmix(word, w, which) + _wmix(flipped, w, which)


def corner_arrays(mesh):
    """(face index, next-corner index) of every corner."""
    off = np.asarray(mesh.face_offsets, dtype=np.int64)
    F = len(off) - 1
    sizes = np.diff(off)
    face = np.repeat(np.arange(F, dtype=np.int64), sizes)
    nxt = np.arange(off[-1], dtype=np.int64) + 1
    last = off[1:] - 1
    nxt[last[sizes > 0]] = off[:-1][sizes > 0]
    return face, nxt


def cycle_hash(mesh) -> np.ndarray:
    """Rotation-invariant, orientation-sensitive hash of each face's edge-plane cycle: the sum of
    mix(e_i, e_{i+1}) over its consecutive (directed) pairs."""
    e = np.asarray(mesh.edge_planes, dtype=np.int64)
    face, nxt = corner_arrays(mesh)
    pair = mix64((e.astype(np.uint64) << np.uint64(32)) ^ e[nxt].astype(np.uint64) ^ np.uint64(0xC1C1E))
    F = len(mesh.face_offsets) - 1
    out = np.zeros(F, dtype=np.uint64)
    with np.errstate(over="ignore"):
        np.add.at(out, face, pair)
    return out


def digest(mesh, N: int) -> dict:
    """Order-independent digests of a mesh: counts, the face-key set (two 64-bit sums), the face
    keys with their edge cycles, and the Euler characteristic."""
    keys = np.ascontiguousarray(mesh.face_keys, dtype=np.uint64)
    h0, h1 = face_hash(keys, 0), face_hash(keys, 1)
    cyc = cycle_hash(mesh)
    with np.errstate(over="ignore"):
        d_keys0 = int(mix64(h0).sum(dtype=np.uint64))
        d_keys1 = int(mix64(h1).sum(dtype=np.uint64))
        d_cycles = int(mix64(h0 ^ mix64(cyc)).sum(dtype=np.uint64))
    F = len(mesh.face_offsets) - 1
    corners = int(mesh.face_offsets[-1])
    open_faces = int(np.count_nonzero(np.add.reduceat((np.asarray(mesh.edge_planes) >= N).astype(np.int64),
                                                      np.asarray(mesh.face_offsets[:-1], dtype=np.int64))
                                      if F else np.zeros(0)))
    return {"faces": F, "corners": corners, "vertices": int(len(mesh.xyz)), "open_faces": open_faces,
            "euler": int(len(mesh.xyz)) - corners // 2 + F if corners % 2 == 0 else None,
            "keys0": f"{d_keys0:016x}", "keys1": f"{d_keys1:016x}", "cycles": f"{d_cycles:016x}"}


def closure(mesh, N: int, strict: bool = True) -> dict:
    """Every neuron edge has its reciprocal (the face of cell key ^ e_p lists plane p), every
    such edge is seen exactly twice, faces have distinct keys, every vertex not on the box is
    used by >= 3 corners.  strict: assert all of it; else return the faces of the edges that
    fail (`unmatched_faces`, indices) and the counts, for the caller to explain (a plane within
    delta of a vertex, counted as a degenerate event, drops an edge shorter than delta from one
    of the two faces that share it)."""
    keys = np.ascontiguousarray(mesh.face_keys, dtype=np.uint64)
    F = keys.shape[0]
    e = np.asarray(mesh.edge_planes, dtype=np.int64)
    face, nxt = corner_arrays(mesh)
    res = {"faces": F, "unmatched_edges": 0, "edges_not_twice": 0}
    bad_faces = set()
    for which in (0, 1):
        h = face_hash(keys, which)
        assert len(np.unique(h)) == F, "two faces share a key fingerprint (duplicate face?)"
        inner = e < N
        f, p = face[inner], e[inner]
        hn = _flip_hash(h, keys, f, p, which)
        # the reciprocal edge instance (neighbour, p) must be among the edge instances
        with np.errstate(over="ignore"):
            mine = mix64(h[f] + mix64(p.astype(np.uint64) + np.uint64(0xED6E)))
            theirs = mix64(hn + mix64(p.astype(np.uint64) + np.uint64(0xED6E)))
        ok = np.isin(theirs, mine)
        if strict:
            assert ok.all(), f"{int((~ok).sum())} neuron edges have no reciprocal face"
        res["unmatched_edges"] = max(res["unmatched_edges"], int((~ok).sum()))
        bad_faces.update(int(x) for x in f[~ok])
        # the neighbour's face, where it exists, is part of the story too
        if not ok.all():
            hs = np.argsort(h)
            pos = np.searchsorted(h[hs], hn[~ok])
            pos = np.minimum(pos, F - 1)
            hit = h[hs][pos] == hn[~ok]
            bad_faces.update(int(x) for x in hs[pos][hit])
        # each undirected edge (unordered face pair, plane) exactly twice
        lo, hi = np.minimum(h[f], hn), np.maximum(h[f], hn)
        with np.errstate(over="ignore"):
            eid = mix64(lo ^ mix64(hi) ^ mix64(p.astype(np.uint64) + np.uint64(0xE1D)))
        u, inv, cnt = np.unique(eid, return_inverse=True, return_counts=True)
        if strict:
            assert np.all(cnt == 2), f"{int((cnt != 2).sum())} edges not shared by exactly two faces"
        res["edges_not_twice"] = max(res["edges_not_twice"], int((cnt != 2).sum()))
        bad_faces.update(int(x) for x in f[cnt[inv] > 2])
        res["neuron_edges"] = int(inner.sum())
    fv = np.asarray(mesh.face_vertices, dtype=np.int64)
    uses = np.bincount(fv, minlength=len(mesh.xyz))
    on_box = np.zeros(len(mesh.xyz), dtype=bool)
    # corner j lies between edge j-1 (the edge whose next corner is j) and edge j
    prev = np.empty_like(nxt)
    prev[nxt] = np.arange(len(nxt))
    box_corner = (e >= N) | (e[prev] >= N)
    on_box[fv[box_corner]] = True
    thin = ~on_box & (uses < 3)
    if strict:
        assert not thin.any(), "a vertex off the box is used by fewer than 3 corners"
    res["thin_vertices"] = int(thin.sum())
    res["box_edges"] = int((e >= N).sum())
    res["unmatched_faces"] = sorted(bad_faces)
    return res


def vertex_key_hash(mesh, N: int, which: int = 0) -> np.ndarray:
    """Hash of each corner's combinatorial vertex key (lo, hi, key with bits lo and hi cleared);
    corner j sits between edge j - 1 and edge j.  Box planes (>= N) clear no bit."""
    keys = np.ascontiguousarray(mesh.face_keys, dtype=np.uint64)
    e = np.asarray(mesh.edge_planes, dtype=np.int64)
    face, nxt = corner_arrays(mesh)
    prev = np.empty_like(nxt)
    prev[nxt] = np.arange(len(nxt))
    a, b = e[prev], e
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    h = face_hash(keys, which)[face]
    one = np.uint64(1)
    with np.errstate(over="ignore"):
        # the word of lo (lo < hi, so hi < N implies lo < N), with hi cleared too when it is there
        sel = np.flatnonzero(lo < N)
        w = lo[sel] >> 6
        word = keys[face[sel], w]
        clr = word & ~(one << (lo[sel] & 63).astype(np.uint64))
        both = (hi[sel] < N) & ((hi[sel] >> 6) == w)
        clr = np.where(both, clr & ~(one << (hi[sel] & 63).astype(np.uint64)), clr)
        h[sel] += _wmix(clr, w, which) - _wmix(word, w, which)
        # the word of hi when it differs from lo's
        sel = np.flatnonzero((hi < N) & ((hi >> 6) != (lo >> 6)))
        w = hi[sel] >> 6
        word = keys[face[sel], w]
        clr = word & ~(one << (hi[sel] & 63).astype(np.uint64))
        h[sel] += _wmix(clr, w, which) - _wmix(word, w, which)
        return mix64(h ^ mix64((lo.astype(np.uint64) << np.uint64(32)) ^ hi.astype(np.uint64)))


def vertex_bijection(mesh, N: int) -> int:
    """The assembled vertex indices are exactly one per combinatorial vertex key: the number of
    distinct keys, of distinct (key, index) pairs and of distinct indices are all the vertex
    count."""
    vk = vertex_key_hash(mesh, N, 0) ^ mix64(vertex_key_hash(mesh, N, 1))
    fv = np.asarray(mesh.face_vertices, dtype=np.int64)
    n_keys = len(np.unique(vk))
    n_pairs = len(np.unique(mix64(vk ^ mix64(fv.astype(np.uint64) + np.uint64(0xB17)))))
    n_idx = len(np.unique(fv))
    assert n_pairs == n_keys, "one vertex key mapped to two vertex indices"
    assert n_pairs == n_idx, "one vertex index holds two vertex keys"
    assert n_idx == len(mesh.xyz), "vertices that no corner uses"
    return n_idx


def face_diff(ma, mb):
    """Faces of mesh a not in b, of b not in a, and common faces whose edge cycles differ (face
    indices into a and b)."""
    ha = face_hash(ma.face_keys, 0) ^ mix64(face_hash(ma.face_keys, 1))
    hb = face_hash(mb.face_keys, 0) ^ mix64(face_hash(mb.face_keys, 1))
    only_a = np.flatnonzero(~np.isin(ha, hb))
    only_b = np.flatnonzero(~np.isin(hb, ha))
    ca, cb = cycle_hash(ma), cycle_hash(mb)
    ia = np.argsort(ha)
    ib = np.argsort(hb)
    common, xa, xb = np.intersect1d(ha[ia], hb[ib], assume_unique=True, return_indices=True)
    fa, fb = ia[xa], ib[xb]
    diff = np.flatnonzero(ca[fa] != cb[fb])
    return only_a, only_b, fa[diff], fb[diff]


class ArrayMesh:
    """The array layout of a mesh (as the C ABI returns it) built from the oracle's faces, with
    vertices assembled by combinatorial key (the oracle's own Mesh.assemble)."""

    def __init__(self, oracle_mesh, N: int):
        faces = oracle_mesh.faces
        kw = (N + 63) // 64
        xyz, idx, _ = oracle_mesh.assemble()
        self.xyz = xyz
        sizes = np.array([len(f.edges) for f in faces], dtype=np.int64)
        self.face_offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.face_vertices = np.concatenate([np.asarray(i, dtype=np.int32) for i in idx]) if faces else \
            np.zeros(0, np.int32)
        self.edge_planes = np.concatenate([np.asarray(f.edges, dtype=np.int32) for f in faces]) if faces else \
            np.zeros(0, np.int32)
        mask = (1 << 64) - 1
        self.face_keys = np.array([[(f.key >> (64 * w)) & mask for w in range(kw)] for f in faces],
                                  dtype=np.uint64).reshape(len(faces), kw)
        self.n_open_faces = oracle_mesh.open_faces()

    @property
    def n_faces(self) -> int:
        return len(self.face_offsets) - 1
