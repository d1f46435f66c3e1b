// am_mesh_host.cu -- host post-processing of a copied-out mesh (no device code, no context).
//
// Canonical order (Alg. 1 leaves the order of the faces to the march; the breadth-first
// discovery on the GPU is not deterministic): faces ascending by cell key as an N-bit
// integer, each face's ring started at its canonical corner, vertices numbered by first
// appearance.  Fan triangulation: the paper notes that every polygon splits into triangles
// along diagonals (Sec. 4.4); a convex face of V corners gives V - 2 triangles fanned from its
// first corner.
#include <algorithm>
#include <numeric>
#include <utility>
#include <vector>

#include "../../include/analytic_marching.h"

namespace {

// the arrays of a host mesh are consistent: offsets rise from 0 to n_corners, vertex indices
// lie in [0, n_vertices), every face has at least three corners
bool mesh_ok(const am_mesh *m)
{
    if (!m || m->n_faces < 0 || m->n_vertices < 0 || m->n_corners < 0 || m->key_words < 1) return false;
    if (m->n_faces == 0) return m->n_corners == 0;
    if (!m->face_offsets || !m->face_vertices || !m->edge_planes || !m->face_keys || (m->n_vertices && !m->xyz))
        return false;
    if (m->face_offsets[0] != 0 || m->face_offsets[m->n_faces] != m->n_corners) return false;
    for (int64_t f = 0; f < m->n_faces; ++f)
        if (m->face_offsets[f + 1] - m->face_offsets[f] < 3) return false;
    for (int64_t c = 0; c < m->n_corners; ++c)
        if (m->face_vertices[c] < 0 || m->face_vertices[c] >= m->n_vertices) return false;
    return true;
}

// corner c of a ring of V corners sits between edge c-1 and edge c: its plane pair, sorted
std::pair<int32_t, int32_t> corner_pair(const int32_t *e, int64_t V, int64_t c)
{
    const int32_t a = e[(c + V - 1) % V], b = e[c];
    return a < b ? std::make_pair(a, b) : std::make_pair(b, a);
}

}  // namespace

extern "C" am_status am_mesh_canonicalize(am_mesh *m)
{
    if (!mesh_ok(m)) return AM_ERR_INVALID_ARG;
    const int64_t F = m->n_faces, K = m->n_corners, NV = m->n_vertices;
    const int kw = m->key_words;
    if (F == 0) return AM_OK;
    const int64_t *off = m->face_offsets;
    const uint64_t *keys = m->face_keys;

    // faces ascending by key: word kw-1 holds the most significant bits
    std::vector<int64_t> order(F);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        for (int w = kw - 1; w >= 0; --w) {
            const uint64_t x = keys[a * kw + w], y = keys[b * kw + w];
            if (x != y) return x < y;
        }
        return false;
    });

    std::vector<int64_t> off2(F + 1);
    std::vector<int32_t> fv2(K), fe2(K);
    std::vector<uint64_t> keys2((size_t)F * kw);
    int64_t c2 = 0;
    for (int64_t i = 0; i < F; ++i) {
        const int64_t f = order[i], b = off[f], V = off[f + 1] - off[f];
        const int32_t *e = m->edge_planes + b;
        int64_t r = 0;
        for (int64_t c = 1; c < V; ++c)
            if (corner_pair(e, V, c) < corner_pair(e, V, r)) r = c;
        off2[i] = c2;
        for (int64_t j = 0; j < V; ++j) {
            fv2[c2 + j] = m->face_vertices[b + (r + j) % V];
            fe2[c2 + j] = e[(r + j) % V];
        }
        c2 += V;
        std::copy(keys + f * kw, keys + (f + 1) * kw, keys2.begin() + i * kw);
    }
    off2[F] = c2;

    // vertices numbered by first appearance; any vertex no face uses keeps its relative order
    // after the used ones
    std::vector<int32_t> id(NV, -1);
    int32_t next = 0;
    for (int64_t c = 0; c < K; ++c)
        if (id[fv2[c]] < 0) id[fv2[c]] = next++;
    for (int64_t v = 0; v < NV; ++v)
        if (id[v] < 0) id[v] = next++;
    std::vector<double> xyz2((size_t)NV * 3);
    for (int64_t v = 0; v < NV; ++v)
        for (int k = 0; k < 3; ++k) xyz2[(size_t)id[v] * 3 + k] = m->xyz[v * 3 + k];
    for (int64_t c = 0; c < K; ++c) fv2[c] = id[fv2[c]];

    std::copy(off2.begin(), off2.end(), m->face_offsets);
    std::copy(fv2.begin(), fv2.end(), m->face_vertices);
    std::copy(fe2.begin(), fe2.end(), m->edge_planes);
    std::copy(keys2.begin(), keys2.end(), m->face_keys);
    std::copy(xyz2.begin(), xyz2.end(), m->xyz);
    return AM_OK;
}

extern "C" am_status am_mesh_triangulate(const am_mesh *m, int32_t *tri, int64_t *n_tri)
{
    if (!n_tri || !mesh_ok(m)) return AM_ERR_INVALID_ARG;
    const int64_t need = m->n_corners - 2 * m->n_faces;
    if (!tri) {
        *n_tri = need;
        return AM_OK;
    }
    if (*n_tri < need) return AM_ERR_CAPACITY;
    int64_t t = 0;
    for (int64_t f = 0; f < m->n_faces; ++f) {
        const int64_t b = m->face_offsets[f], V = m->face_offsets[f + 1] - b;
        for (int64_t j = 1; j + 1 < V; ++j, ++t) {
            tri[3 * t + 0] = m->face_vertices[b];
            tri[3 * t + 1] = m->face_vertices[b + j];
            tri[3 * t + 2] = m->face_vertices[b + j + 1];
        }
    }
    *n_tri = need;
    return AM_OK;
}
