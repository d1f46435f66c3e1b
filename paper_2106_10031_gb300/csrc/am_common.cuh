// am_common.cuh -- device-side data layout shared by the library's kernels.
//
// Cells, keys and faces live in flat arenas indexed by a cell id.  Ids are handed out in
// the order cells are discovered; the march solves them in id order (first in, first out),
// so the id range [solved, allocated) is Alg. 1's active set S* and every id ever handed
// out, indexed by the hash table, is S* u S.
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

// indices into the device counter array.  Every counter sits on its own 128-byte line
// (a stride of 16 words) so that the ticket counters polled by waiting blocks do not share a
// line with the counters every solved cell updates.
constexpr int kCtrStride = 16;
enum {
    kNCells = 0 * kCtrStride,       // cell ids handed out
    kStatus = 1 * kCtrStride,       // sticky status bits
    kDegenerate = 2 * kCtrStride,   // planes within delta of accepted vertices
    kEmpty = 3 * kCtrStride,        // cells whose face was empty / of zero area
    kSolved = 4 * kCtrStride,       // cells solved
    kRefined = 5 * kCtrStride,      // mixed precision: cells redone in FP64
    kHead = 6 * kCtrStride,         // next queue ticket (persistent schedule)
    kDone = 7 * kCtrStride,         // tickets finished (solved, dead or skipped)
    kCloseCalls = 8 * kCtrStride,   // mixed precision: sign tests re-evaluated in FP64
    kFixups = 9 * kCtrStride,       // faces whose candidate polygon the full check corrected
    kPhase0 = 10 * kCtrStride,      // 10 per-phase cycle counters (timing builds only)
    kCuts = 20 * kCtrStride,        // half-plane cuts applied to candidate polygons (clip work)
    kWarpFallback = 21 * kCtrStride,  // cells the warp clip handed to the block kernel
    kNumCounters = 22 * kCtrStride
};

// One loaded network, folded for the device (row-major):
//   pre_l = AT_l^T h_{l-1} + Cl_l [x; 1]
// AT_l (l >= 2) is the hidden part of W_l transposed, n_{l-1} x n_l; Cl_l (n_l x 4) is the
// cell-independent affine part: [W_1 | b_1 + W_1^z z] at layer 1, [W^x | b + W^z z] at the
// skip layer, [0 | b_l] elsewhere.  Every array exists in FP64 and as a double-float pair
// (hi = fl32(x), lo = fl32(x - hi)).
struct NetDev {
    int L, N, kw;
    int width[kMaxLayers + 1];   // 1..L
    int row0[kMaxLayers + 1];    // id of the first neuron of layer l
    const double *AT[kMaxLayers + 1];
    const double *Cl[kMaxLayers + 1];
    const float *AThi[kMaxLayers + 1], *ATlo[kMaxLayers + 1];
    const float *Clhi[kMaxLayers + 1], *Cllo[kMaxLayers + 1];
    const double *w_out;
    const float *w_out_hi, *w_out_lo;
    double b_out;
    // tensor-core compose: W_l (hidden part) as three BF16 parts (hi, mid, lo) in mma.m16n8k16
    // A-fragment order, tile (mt, kt) at (mt * Kt + kt) * 96 uint4 (32 lanes per part), and the
    // per row m of W_l the pair (|W_m|_2, max_j |W_mj|)
    const uint4 *Wf[kMaxLayers + 1];
    const float *wn[kMaxLayers + 1];
    unsigned long long salt;     // per-net hash salt
    int df_ok;                   // 1: the double-float bound stays useful through this net's depth
    double slope;                // hidden activation a (a > 0), slope a (a <= 0); 0 = ReLU
    // residual shortcuts from hidden layers (Sec. 5.1): layer l adds S_l h_{sc_src[l]} (sc_src 0 =
    // none; a shortcut from x is folded into Cl); sc_S[l] = S_l (n_l x n_src) or null = identity
    int sc_src[kMaxLayers + 1];
    const double *sc_S[kMaxLayers + 1];
    int fp64_only;               // 1: composes in FP64 only (leaky activation, a hidden shortcut, pooling)
    // final max pooling over M heads (Sec. 5.2); M = 0 for a single output.  The units are rows
    // 0 .. n_units - 1, the pooling rows (and one-hot key bits of the pooled index) n_units .. N - 1
    int M, n_units;
    const double *w_heads;       // M x n_L
    const double *b_heads;       // M
};

// The pooled index j of a cell of a pooled net: the one-hot key bit among n_units .. N - 1
__device__ __forceinline__ int pooled_index(const NetDev &net, const unsigned long long *key)
{
    for (int i = 0; i < net.M; ++i) {
        const int b = net.n_units + i;
        if ((key[b >> 6] >> (b & 63)) & 1ull) return i;
    }
    return 0;
}

// Device arenas (all sized at context creation).
struct Arena {
    unsigned long long *keys;    // cap x kw
    int32_t *net;                // cap
    unsigned long long *hash;    // cap (Zobrist hash of the key, salted by the net)
    int32_t *nverts;             // cap: corners of the cell's face (0 = empty, -1 unsolved, -2 dead)
    int32_t *edges;              // cap x maxv: plane of edge i -> i+1
    double *verts;               // cap x maxv x 3
    unsigned *ready;             // cap: 1 once the cell's record is written (persistent schedule)
    int32_t *entry_plane;        // cap: plane crossed to reach the cell (-1 for a seed)
    float *entry_pt;             // cap x 3: a point of the face (edge midpoint or seed point)
    int32_t *parent;             // cap: the cell whose push created this one (-1 for a seed)
    int32_t *chain;              // cap: rank-1 composes since the last full compose (sliced level march)
    int32_t *cls;                // cap: sliced level march, per cell of the next level: -1 full compose,
                                 //      else the layer of the flipped neuron (rank-1 compose from the parent)
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
