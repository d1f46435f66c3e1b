// am_common.cuh -- device-side data layout shared by the library's kernels.
//
// Cells, keys and faces live in flat arenas indexed by a cell id.  Ids are handed out in
// the order cells are discovered, so the cells found while solving breadth-first level i
// form the contiguous id range of level i + 1 (Alg. 1's active set S* is a range of ids;
// S. the set of all ids handed out so far, indexed by the hash table).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace am {

constexpr int kMaxLayers = 32;
constexpr int kBoxPlanes = 6;      // ids N + 0..5 : +x, -x, +y, -y, +z, -z
constexpr int kSquarePlanes = 4;   // ids N + 6..9 : the initial square, always clipped away
constexpr uint32_t kNoFlip = 0x1FFFu;          // 13-bit "no flipped neuron" in a hash-slot ref
constexpr int kMaxNeurons = 8190;              // neuron ids must fit the 13-bit flip field
constexpr int64_t kMaxCellIds = (int64_t)1 << 27;  // 27-bit parent field of a slot ref

// status bits (sticky, OR-ed into counters[kStatus])
enum : unsigned long long {
    kStCellCap = 1ull,      // cell arena full
    kStHashFull = 2ull,     // cell hash table probe limit hit
    kStFaceVerts = 4ull,    // a face needed more than max_face_verts corners
    kStVertHash = 8ull,     // vertex hash table probe limit hit
    kStSeedNoSign = 16ull,  // a seed ray had no sign change
    kStSeedNoCell = 32ull,  // a seed ray's bisection found no common cell
    kStTimeout = 64ull,     // a bounded device wait gave up
    kStClip = 128ull,       // a clip step met an inconsistent polygon
};

// indices into the device counter array
enum {
    kNCells = 0,        // cell ids handed out
    kStatus = 1,        // sticky status bits
    kDegenerate = 2,    // planes within delta of accepted vertices
    kEmpty = 3,         // cells whose face was empty / of zero area
    kSolved = 4,        // cells solved
    kRefined = 5,       // mixed precision: cells redone in FP64
    kNumCounters = 16
};

// One loaded network, folded for the device (row-major, FP64):
//   pre_l = AT_l^T h_{l-1} + Cl_l [x; 1]
// AT_l (l >= 2) is the hidden part of W_l transposed, n_{l-1} x n_l; Cl_l (n_l x 4) is the
// cell-independent affine part: [W_1 | b_1 + W_1^z z] at layer 1, [W^x | b + W^z z] at the
// skip layer, [0 | b_l] elsewhere.
struct NetDev {
    int L, N, kw;
    int width[kMaxLayers + 1];   // 1..L
    int row0[kMaxLayers + 1];    // id of the first neuron of layer l
    const double *AT[kMaxLayers + 1];
    const double *Cl[kMaxLayers + 1];
    const double *w_out;
    double b_out;
    unsigned long long salt;     // per-net hash salt
};

// Device arenas (all sized at context creation).
struct Arena {
    unsigned long long *keys;    // cap x kw
    int32_t *net;                // cap
    unsigned long long *hash;    // cap (Zobrist hash of the key, salted by the net)
    int32_t *nverts;             // cap: corners of the cell's face (0 = empty)
    int32_t *edges;              // cap x maxv: plane of edge i -> i+1
    double *verts;               // cap x maxv x 3
    unsigned long long *slots;   // cell hash table
    unsigned long long slot_mask;
    const unsigned long long *zob;   // Zobrist table, one 64-bit value per neuron id
    unsigned long long *counters;    // kNumCounters
    int kw;
    int maxv;
    int64_t cap;
};

// ---- hash-slot encoding: [63] 1 | [62:40] tag (23 bits) | [39:13] parent cell | [12:0] flip
__host__ __device__ inline unsigned long long slot_make(unsigned long long h, unsigned long long parent,
                                                        unsigned flip)
{
    return (1ull << 63) | (((h >> 41) & 0x7FFFFFull) << 40) | ((parent & 0x7FFFFFFull) << 13) | (flip & 0x1FFFu);
}
__host__ __device__ inline unsigned long long slot_tag(unsigned long long s) { return (s >> 40) & 0x7FFFFFull; }
__host__ __device__ inline unsigned long long hash_tag(unsigned long long h) { return (h >> 41) & 0x7FFFFFull; }
__host__ __device__ inline int64_t slot_parent(unsigned long long s) { return (int64_t)((s >> 13) & 0x7FFFFFFull); }
__host__ __device__ inline unsigned slot_flip(unsigned long long s) { return (unsigned)(s & 0x1FFFu); }

// splitmix64 (Steele, Lea & Flood 2014): the Zobrist table and the net salts.
__host__ __device__ inline unsigned long long splitmix64(unsigned long long x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

}  // namespace am
