// am_noalloc.cu -- vertex deduplication that allocates nothing.
//
// Callers that must not allocate device memory get this entry point.  That covers code
// running inside a CUDA graph capture, inside a host framework that owns every device
// allocation through its own pool, or under a fixed memory budget.  It is the deduplication
// step of the mesh assembly (the combinatorial vertex key (i, j, s with bits i and j
// cleared)) as a standalone call: the caller passes the faces and the output array, and the
// only scratch memory is the file-scope table below.  That table holds kNoAllocSlots 64-bit
// slots (32 MiB) and one counter; every GPU that loads the library keeps it until the
// process exits.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/analytic_marching.h"

namespace {

constexpr int64_t kNoAllocSlots = (int64_t)1 << 22;          // hash slots (load factor <= 1/2)
constexpr int64_t kNoAllocMaxCorners = kNoAllocSlots / 2;    // AM_NOALLOC_MAX_CORNERS
constexpr int kNoAllocMaxFaceCorners = 62;                   // AM_NOALLOC_MAX_FACE_CORNERS (6-bit corner field)
constexpr int kNoAllocMaxDevices = 64;
constexpr int kNoAllocProbe = 1 << 16;
constexpr int32_t kWin = 1 << 30;

// slots [0, kNoAllocSlots), the vertex counter at [kNoAllocSlots] and the error bits at
// [kNoAllocSlots + 1]: 1 = a face with more than kNoAllocMaxFaceCorners corners or with offsets
// outside [0, n_corners], 2 = a corner whose vertex could not be found or claimed (probe limit)
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocSlots + 32];
constexpr unsigned long long kErrFace = 1ull, kErrProbe = 2ull;

std::mutex g_setup_mutex;
void *g_scratch_addr[kNoAllocMaxDevices] = {};

__device__ __forceinline__ unsigned long long mix64(unsigned long long x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

struct NoAllocArgs {
    const unsigned long long *keys;
    int kw;
    const int64_t *off;
    const int32_t *planes;
    int64_t n_faces;
    int64_t n_corners;
    int n_neurons;
    int32_t *out;
    unsigned long long *slots;
    unsigned long long mask;
};

__device__ __forceinline__ void corner_pair(const NoAllocArgs &a, int64_t f, int j, int *lo, int *hi)
{
    const int64_t b = a.off[f];
    const int m = (int)(a.off[f + 1] - b);
    const int p = a.planes[b + (j + m - 1) % m], q = a.planes[b + j];
    *lo = p < q ? p : q;
    *hi = p < q ? q : p;
}

__device__ __forceinline__ unsigned long long masked_word(const NoAllocArgs &a, int64_t f, int w, int lo, int hi)
{
    unsigned long long x = a.keys[f * a.kw + w];
    if (lo < a.n_neurons && (lo >> 6) == w) x &= ~(1ull << (lo & 63));
    if (hi < a.n_neurons && (hi >> 6) == w) x &= ~(1ull << (hi & 63));
    return x;
}

__device__ unsigned long long corner_hash(const NoAllocArgs &a, int64_t f, int lo, int hi)
{
    unsigned long long h = mix64(((unsigned long long)lo << 20) ^ (unsigned long long)hi);
    for (int w = 0; w < a.kw; ++w) h = mix64(h ^ masked_word(a, f, w, lo, hi));
    return h;
}

__device__ bool same_vertex(const NoAllocArgs &a, int64_t f, int64_t g, int lo, int hi)
{
    for (int w = 0; w < a.kw; ++w)
        if (masked_word(a, f, w, lo, hi) != masked_word(a, g, w, lo, hi)) return false;
    return true;
}

// slot: [63] 1 | [62:40] tag | [39:6] face | [5:0] corner
__device__ unsigned long long probe(const NoAllocArgs &a, int64_t f, int j, bool claim, bool *claimed)
{
    int lo, hi;
    corner_pair(a, f, j, &lo, &hi);
    const unsigned long long h = corner_hash(a, f, lo, hi);
    const unsigned long long mine = (1ull << 63) | (((h >> 41) & 0x7FFFFFull) << 40) |
                                    (((unsigned long long)f & 0x3FFFFFFFFull) << 6) | ((unsigned long long)j & 63ull);
    unsigned long long pos = h & a.mask;
    *claimed = false;
    for (int i = 0; i < kNoAllocProbe; ++i) {
        unsigned long long cur = *((volatile unsigned long long *)(a.slots + pos));
        if (cur == 0ull && claim) {
            cur = atomicCAS(a.slots + pos, 0ull, mine);
            if (cur == 0ull) { *claimed = true; return mine; }
        }
        if (cur == 0ull) return 0ull;
        if (((cur >> 40) & 0x7FFFFFull) == ((h >> 41) & 0x7FFFFFull)) {
            const int64_t g = (int64_t)((cur >> 6) & 0x3FFFFFFFFull);
            if (g >= a.n_faces) return 0ull;          // never written by this call: not a slot of ours
            int lo2, hi2;
            corner_pair(a, g, (int)(cur & 63), &lo2, &hi2);
            if (lo2 == lo && hi2 == hi && same_vertex(a, f, g, lo, hi)) return cur;
        }
        pos = (pos + 1) & a.mask;
    }
    return 0ull;
}

// a face whose corners this call can key: offsets inside [0, n_corners] and at most
// kNoAllocMaxFaceCorners corners (the slot's 6-bit corner field)
__device__ __forceinline__ bool face_ok(const NoAllocArgs &a, int64_t f, int64_t *b, int *m)
{
    const int64_t b0 = a.off[f], b1 = a.off[f + 1];
    *b = b0;
    *m = (int)(b1 - b0);
    return b0 >= 0 && b1 >= b0 && b1 <= a.n_corners && b1 - b0 <= kNoAllocMaxFaceCorners;
}

__global__ void noalloc_insert_kernel(NoAllocArgs a)
{
    unsigned long long *count = g_noalloc_scratch + kNoAllocSlots;
    unsigned long long *err = g_noalloc_scratch + kNoAllocSlots + 1;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < a.n_faces; f += (int64_t)gridDim.x * blockDim.x) {
        int64_t b;
        int m;
        if (!face_ok(a, f, &b, &m)) {
            // no slot names this face; a face that is only too long gets -1 at its corners (rising
            // offsets tile [0, n_corners] without overlap, so these writes stay within n_corners)
            atomicOr(err, kErrFace);
            if (b >= 0 && m > 0 && b + m <= a.n_corners)
                for (int j = 0; j < m; ++j) a.out[b + j] = -1;
            continue;
        }
        for (int j = 0; j < m; ++j) {
            bool claimed;
            probe(a, f, j, true, &claimed);
            a.out[b + j] = claimed ? ((int32_t)atomicAdd(count, 1ull) | kWin) : -1;
        }
    }
}

__global__ void noalloc_lookup_kernel(NoAllocArgs a)
{
    unsigned long long *err = g_noalloc_scratch + kNoAllocSlots + 1;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < a.n_faces; f += (int64_t)gridDim.x * blockDim.x) {
        int64_t b;
        int m;
        if (!face_ok(a, f, &b, &m)) continue;          // reported by the insert kernel
        for (int j = 0; j < m; ++j) {
            const int32_t v = a.out[b + j];
            if (v != -1) { a.out[b + j] = v & ~kWin; continue; }
            bool claimed;
            const unsigned long long s = probe(a, f, j, false, &claimed);
            if (s == 0ull) {              // not found (a probe gave up): stays -1, the count goes negative
                atomicOr(err, kErrProbe);
                continue;
            }
            const int64_t g = (int64_t)((s >> 6) & 0x3FFFFFFFFull);
            a.out[b + j] = a.out[a.off[g] + (int)(s & 63)] & ~kWin;
        }
    }
}

// the vertex count, or minus the error bits when some corner was left without a vertex
__global__ void noalloc_count_kernel(int64_t *n_out)
{
    const unsigned long long e = g_noalloc_scratch[kNoAllocSlots + 1];
    *n_out = e ? -(int64_t)e : (int64_t)g_noalloc_scratch[kNoAllocSlots];
}

}  // namespace

extern "C" am_status am_assign_vertices_noalloc(const uint64_t *d_face_keys, int key_words,
                                                const int64_t *d_face_offsets, const int32_t *d_edge_planes,
                                                int64_t n_faces, int64_t n_corners, int n_neurons,
                                                int32_t *d_corner_vertex, int64_t *d_n_vertices, void *stream)
{
    if (!d_face_keys || !d_face_offsets || !d_edge_planes || !d_corner_vertex || !d_n_vertices || key_words < 1 ||
        n_faces < 0 || n_corners < 0 || n_neurons < 1 || n_faces >= ((int64_t)1 << 34))
        return AM_ERR_INVALID_ARG;
    if (n_corners > kNoAllocMaxCorners) return AM_ERR_CAPACITY;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return AM_ERR_CUDA;
    void *scratch = nullptr;
    {
        // once per device, with that device current: the device address of the static table
        // (in host code the symbol itself only names a host-side stand-in)
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return AM_ERR_CUDA;
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    int64_t slots = 1024;
    while (slots < 2 * n_corners) slots <<= 1;
    unsigned long long *tab = (unsigned long long *)scratch;
    // the table keeps the previous call's contents: clear the part in use, the counter and the
    // error bits
    if (cudaMemsetAsync(tab, 0, sizeof(unsigned long long) * slots, st) != cudaSuccess) return AM_ERR_CUDA;
    if (cudaMemsetAsync(tab + kNoAllocSlots, 0, 2 * sizeof(unsigned long long), st) != cudaSuccess) return AM_ERR_CUDA;
    if (n_faces == 0) {
        if (cudaMemsetAsync(d_n_vertices, 0, sizeof(int64_t), st) != cudaSuccess) return AM_ERR_CUDA;
        return AM_OK;
    }
    NoAllocArgs a{};
    a.keys = (const unsigned long long *)d_face_keys;
    a.kw = key_words;
    a.off = d_face_offsets;
    a.planes = d_edge_planes;
    a.n_faces = n_faces;
    a.n_corners = n_corners;
    a.n_neurons = n_neurons;
    a.out = d_corner_vertex;
    a.slots = tab;
    a.mask = (unsigned long long)(slots - 1);
    int64_t g = (n_faces + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    noalloc_insert_kernel<<<(unsigned)g, 256, 0, st>>>(a);
    noalloc_lookup_kernel<<<(unsigned)g, 256, 0, st>>>(a);
    noalloc_count_kernel<<<1, 1, 0, st>>>(d_n_vertices);
    return cudaGetLastError() == cudaSuccess ? AM_OK : AM_ERR_CUDA;
}
