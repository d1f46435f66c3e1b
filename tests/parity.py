"""Comparison of a mesh from the CUDA path with the oracle's, element by element.

Both sides are brought to the same canonical form: per face its cell key, the cyclic list
of edge planes CCW about +grad F starting at the vertex whose sorted plane pair is
smallest, and the matching vertex coordinates.  Face keys and edge cycles must be equal
(bit exact); coordinates agree within a relative tolerance; the assembled vertex indices
must coincide exactly with the combinatorial vertex keys.
"""
from __future__ import annotations

import numpy as np


def _key_int(words) -> int:
    return int.from_bytes(np.asarray(words, dtype=np.uint64).tobytes(), "little")


def canon(edges, verts):
    m = len(edges)
    pairs = [(min(edges[j - 1], edges[j]), max(edges[j - 1], edges[j])) for j in range(m)]
    j0 = min(range(m), key=lambda j: pairs[j])
    return [int(e) for e in edges[j0:]] + [int(e) for e in edges[:j0]], np.roll(np.asarray(verts), -j0, axis=0)


def gpu_faces(mesh):
    """{key: (edges, verts (m x 3), vertex indices)} from a paper_2106_10031_gb300.Mesh."""
    out = {}
    o = mesh.face_offsets
    for i in range(mesh.n_faces):
        idx = mesh.face_vertices[o[i]:o[i + 1]]
        e = mesh.edge_planes[o[i]:o[i + 1]]
        k = _key_int(mesh.face_keys[i])
        assert k not in out, "duplicate face key"
        m = len(e)
        pairs = [(min(e[j - 1], e[j]), max(e[j - 1], e[j])) for j in range(m)]
        j0 = min(range(m), key=lambda j: pairs[j])
        out[k] = ([int(x) for x in np.roll(e, -j0)], mesh.xyz[np.roll(idx, -j0)], np.roll(idx, -j0))
    return out


def vertex_key(key, a, b, N):
    lo, hi = min(a, b), max(a, b)
    k = key
    for p in (lo, hi):
        if p < N:
            k &= ~(1 << p)
    return (lo, hi, k)


def compare(oracle_mesh, gpu_mesh, N, rtol=1e-9, sample=None):
    """Assert parity; returns a dict of measured errors."""
    ref = {f.key: f for f in oracle_mesh.faces}
    got = gpu_faces(gpu_mesh)
    missing = set(ref) - set(got)
    extra = set(got) - set(ref)
    assert not missing and not extra, f"face key sets differ: {len(missing)} missing, {len(extra)} extra"
    keys = sorted(ref)
    if sample is not None and sample < len(keys):
        rng = np.random.default_rng(0)
        keys = [keys[i] for i in rng.choice(len(keys), sample, replace=False)]
    max_rel = 0.0
    for k in keys:
        f = ref[k]
        e_g, v_g, _ = got[k]
        assert f.edges == e_g, f"edge cycle differs for face {k:#x}: {f.edges} vs {e_g}"
        err = np.linalg.norm(f.verts - v_g, axis=1) / np.maximum(1.0, np.linalg.norm(f.verts, axis=1))
        max_rel = max(max_rel, float(err.max()))
    assert max_rel <= rtol, f"vertex error {max_rel:.3e} > {rtol:.1e}"
    # connectivity: GPU vertex index <-> combinatorial vertex key is a bijection
    idx_of = {}
    for k, (e, _, idx) in got.items():
        m = len(e)
        for j in range(m):
            vk = vertex_key(k, e[j - 1], e[j], N)
            i = int(idx[j])
            assert idx_of.setdefault(vk, i) == i, "one vertex key mapped to two vertex indices"
    assert len(set(idx_of.values())) == len(idx_of) == len(gpu_mesh.xyz), "vertex indices are not one per key"
    return {"faces": len(ref), "vertices": len(idx_of), "max_rel_vertex_err": max_rel}


def closure(gpu_mesh, N):
    """Completeness without the oracle: every edge on a neuron plane has its reciprocal
    face (cell ^ e_k, same plane) in the set (Thm. 1 / Alg. 1 steps 10-11), and every
    vertex is shared by at least 3 corners unless it lies on the box."""
    got = gpu_faces(gpu_mesh)
    for k, (e, _, _) in got.items():
        for p in e:
            if p < N:
                g = got.get(k ^ (1 << p))
                assert g is not None and p in g[0], f"edge {p} of face {k:#x} has no reciprocal"
    uses = np.bincount(gpu_mesh.face_vertices, minlength=len(gpu_mesh.xyz))
    on_box = np.zeros(len(gpu_mesh.xyz), dtype=bool)
    o = gpu_mesh.face_offsets
    for i in range(gpu_mesh.n_faces):
        e = gpu_mesh.edge_planes[o[i]:o[i + 1]]
        idx = gpu_mesh.face_vertices[o[i]:o[i + 1]]
        for j in range(len(e)):
            if e[j - 1] >= N or e[j] >= N:
                on_box[idx[j]] = True
    assert np.all(uses[~on_box] >= 3)
    return len(got)


def face_at(mesh, i):
    """(key int, canonical edge cycle, matching vertices) of face i of a binding Mesh."""
    o = mesh.face_offsets
    e = mesh.edge_planes[o[i]:o[i + 1]]
    idx = mesh.face_vertices[o[i]:o[i + 1]]
    edges, verts = canon(e, mesh.xyz[idx])
    return _key_int(mesh.face_keys[i]), edges, verts


def compare_sampled(oracle_mod, net, gpu_mesh, N, sample, rtol, box, seed=0):
    """Each sampled GPU face (uniform over the mesh's faces, hence over every breadth-first
    level) is re-solved by the oracle (Alg. 2 from the nearest line to the GPU face's
    centroid) and must match exactly (edges) and within rtol (vertices).  Touches only the
    sampled faces, so it scales to meshes of millions of faces."""
    rng = np.random.default_rng(seed)
    F = gpu_mesh.n_faces
    pick = rng.choice(F, min(sample, F), replace=False)
    worst = 0.0
    for i in pick:
        k, e_g, v_g = face_at(gpu_mesh, int(i))
        f, rc = oracle_mod.solve_cell(net, k, None, v_g.mean(0), box)
        assert rc == 0 and f is not None, f"oracle could not clip face {k:#x}"
        assert f.edges == e_g, f"edge cycle differs for face {k:#x}: {f.edges} vs {e_g}"
        err = np.linalg.norm(f.verts - v_g, axis=1) / np.maximum(1.0, np.linalg.norm(f.verts, axis=1))
        worst = max(worst, float(err.max()))
    assert worst <= rtol, worst
    return worst
