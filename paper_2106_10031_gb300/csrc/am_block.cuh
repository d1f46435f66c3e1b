// am_block.cuh -- block-wide primitives (scan, compaction, reductions) and the cell
// hash-table insert used by the marching kernels.
#pragma once

#include "am_common.cuh"

namespace am {

constexpr int kMaxProbe = 1 << 16;   // hash probe limit per insert (a bounded loop)

// Exclusive block scan of one int per thread.  wsum: shared scratch of 32 ints.  Every
// thread of the block must call it.  *total receives the block sum.
__device__ __forceinline__ int block_scan_excl(int v, int *wsum, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) wsum[lane] = s;
    }
    __syncthreads();
    const int base = wid ? wsum[wid - 1] : 0;
    *total = wsum[nw - 1];
    __syncthreads();
    return base + x - v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block argmax of (value, index): the larger value wins, ties go to the smaller index.
// idx < 0 marks "no candidate".  red_v/red_i: shared scratch of 32 entries each.
__device__ __forceinline__ void block_argmax(double v, int idx, double *red_v, int *red_i, double *out_v,
                                             int *out_i)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        bool take = (i2 >= 0) && (idx < 0 || v2 > v || (v2 == v && i2 < idx));
        if (take) { v = v2; idx = i2; }
    }
    if (lane == 0) { red_v[wid] = v; red_i[wid] = idx; }
    __syncthreads();
    if (wid == 0) {
        v = lane < nw ? red_v[lane] : 0.0;
        idx = lane < nw ? red_i[lane] : -1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double v2 = __shfl_xor_sync(0xffffffffu, v, o);
            int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
            bool take = (i2 >= 0) && (idx < 0 || v2 > v || (v2 == v && i2 < idx));
            if (take) { v = v2; idx = i2; }
        }
        if (lane == 0) { red_v[0] = v; red_i[0] = idx; }
    }
    __syncthreads();
    *out_v = red_v[0];
    *out_i = red_i[0];
    __syncthreads();
}

constexpr int kNoPool = 1 << 30;       // pooling bit range of a net without pooling

// Word w of the key reached from key word x by crossing plane `flip` (kNoFlip: none).  A unit's
// plane flips its bit (Alg. 1 step 10); a pooling plane of a max-pooled net (pool0 <= flip < pool1,
// Sec. 5.2) moves the one-hot pooled index, bits pool0 .. pool1 - 1, to flip.
__device__ __forceinline__ unsigned long long child_word(unsigned long long x, int w, unsigned flip, int pool0,
                                                         int pool1)
{
    if (flip == kNoFlip) return x;
    if ((int)flip >= pool0 && (int)flip < pool1) {
        const int lo = max(pool0 - 64 * w, 0), hi = min(pool1 - 64 * w, 64);
        if (lo < hi) x &= ~((hi >= 64 ? ~0ull : ((1ull << hi) - 1ull)) & ~((1ull << lo) - 1ull));
        if ((int)(flip >> 6) == w) x |= 1ull << (flip & 63);
        return x;
    }
    if ((int)(flip >> 6) == w) x ^= 1ull << (flip & 63);
    return x;
}

// key(pa) crossed at fa == key(pb) crossed at fb ?  (kNoFlip = nothing crossed)
// Keys written by other blocks of a running kernel are read through L2 (ld.global.cg): the
// SM's L1 is not coherent with other SMs' writes and may hold a stale copy of the line.
__device__ __forceinline__ bool ref_keys_equal(const Arena &ar, int64_t pa, unsigned fa, int64_t pb, unsigned fb,
                                               int pool0 = kNoPool, int pool1 = kNoPool)
{
    const unsigned long long *ka = ar.keys + pa * ar.kw, *kb = ar.keys + pb * ar.kw;
    for (int w = 0; w < ar.kw; ++w) {
        const unsigned long long x = child_word(__ldcg(ka + w), w, fa, pool0, pool1) ^
                                     child_word(__ldcg(kb + w), w, fb, pool0, pool1);
        if (x) return false;
    }
    return true;
}

// Alg. 1 steps 10-11: the neighbour across plane `flip` (hash h) is pushed unless it was seen
// before.  The slot records (parent, flip), from which any later probe rebuilds the key, so a
// claim never waits for a key to be written.  A claim hands out the next cell id, writes the
// new cell's record there (key, net, hash, the crossed plane as the new cell names it, entry,
// or flip when entry < 0, and a point of the shared edge), then publishes it through ready[id].
// pool0, pool1: the pooling bits of a max-pooled net (child_word).
__device__ __forceinline__ void insert_neighbor(const Arena &ar, const unsigned *mask, int64_t parent, int net,
                                                unsigned flip, unsigned long long h, float px, float py, float pz,
                                                int pool0 = kNoPool, int pool1 = kNoPool, int entry = -1)
{
    const unsigned long long mine = slot_make(h, (unsigned long long)parent, flip);
    unsigned long long pos = h & ar.slot_mask;
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        const unsigned long long cur = atomicCAS(ar.slots + pos, 0ull, mine);
        if (cur == 0ull) {
            long long id = (long long)atomicAdd(ar.counters + kNCells, 1ull);
            if (id >= ar.cap) {
                atomicOr(ar.counters + kStatus, kStCellCap);
                return;
            }
            // the parent's key is its state, held by the block in shared memory
            unsigned long long *kn = ar.keys + id * ar.kw;
            for (int w = 0; w < ar.kw; ++w) {
                const unsigned long long x = (unsigned long long)mask[2 * w] | ((unsigned long long)mask[2 * w + 1] << 32);
                kn[w] = child_word(x, w, flip, pool0, pool1);
            }
            ar.net[id] = net;
            ar.hash[id] = h;
            ar.nverts[id] = -1;
            ar.entry_plane[id] = entry >= 0 ? entry : (int32_t)flip;
            ar.parent[id] = (int32_t)parent;
            ar.entry_pt[id * 3 + 0] = px;
            ar.entry_pt[id * 3 + 1] = py;
            ar.entry_pt[id * 3 + 2] = pz;
            // publish: every write above is visible to whoever acquires the flag
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(ar.ready + id), "r"(1u) : "memory");
            return;
        }
        if (slot_tag(cur) == hash_tag(h)) {
            const int64_t pb = slot_parent(cur);
            if (__ldcg(ar.net + pb) == net && ref_keys_equal(ar, parent, flip, pb, slot_flip(cur), pool0, pool1))
                return;
        }
        pos = (pos + 1) & ar.slot_mask;
    }
    atomicOr(ar.counters + kStatus, kStHashFull);
}

// The same push by a whole warp (every lane calls it with the same arguments): lane 0 claims
// the slot and the id, the lanes copy and compare the key words in parallel.  For wide keys
// (N = 4096: 64 words) this turns 2 kw serial L2 round trips per tag hit into 2 kw / 32.
// publish = false (the level schedule: the new cell is read only by later launches, after this
// kernel has ended) skips the fence and the release store that a persistent consumer needs.
__device__ __forceinline__ void insert_neighbor_warp(const Arena &ar, const unsigned *mask, int64_t parent, int net,
                                                     unsigned flip, unsigned long long h, float px, float py,
                                                     float pz, bool publish = true, int pool0 = kNoPool,
                                                     int pool1 = kNoPool, int entry = -1)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long mine = slot_make(h, (unsigned long long)parent, flip);
    unsigned long long pos = h & ar.slot_mask;
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        unsigned long long cur = 0ull;
        if (lane == 0) cur = atomicCAS(ar.slots + pos, 0ull, mine);
        cur = __shfl_sync(0xffffffffu, cur, 0);
        if (cur == 0ull) {
            long long id = 0;
            if (lane == 0) id = (long long)atomicAdd(ar.counters + kNCells, 1ull);
            id = __shfl_sync(0xffffffffu, id, 0);
            if (id >= ar.cap) {
                if (lane == 0) atomicOr(ar.counters + kStatus, kStCellCap);
                return;
            }
            // the parent's key is its state, held by the block in shared memory
            unsigned long long *kn = ar.keys + id * ar.kw;
            for (int w = lane; w < ar.kw; w += 32) {
                const unsigned long long x = (unsigned long long)mask[2 * w] | ((unsigned long long)mask[2 * w + 1] << 32);
                kn[w] = child_word(x, w, flip, pool0, pool1);
            }
            if (lane == 0) {
                ar.net[id] = net;
                ar.hash[id] = h;
                ar.nverts[id] = -1;
                ar.entry_plane[id] = entry >= 0 ? entry : (int32_t)flip;
                ar.parent[id] = (int32_t)parent;
                ar.entry_pt[id * 3 + 0] = px;
                ar.entry_pt[id * 3 + 1] = py;
                ar.entry_pt[id * 3 + 2] = pz;
            }
            if (publish) {
                __threadfence();      // every lane's key words are visible device-wide ...
                __syncwarp();
                // ... before the flag that publishes them
                if (lane == 0) asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(ar.ready + id), "r"(1u) : "memory");
            } else if (lane == 0) {
                ar.ready[id] = 1u;    // visible to later launches at the kernel boundary
            }
            return;
        }
        if (slot_tag(cur) == hash_tag(h)) {
            const int64_t pb = slot_parent(cur);
            const unsigned fb = slot_flip(cur);
            if (__ldcg(ar.net + pb) == net) {
                const unsigned long long *ka = ar.keys + parent * ar.kw, *kb = ar.keys + pb * ar.kw;
                bool diff = false;
                for (int w = lane; w < ar.kw; w += 32) {
                    const unsigned long long x = child_word(__ldcg(ka + w), w, flip, pool0, pool1) ^
                                                 child_word(__ldcg(kb + w), w, fb, pool0, pool1);
                    diff |= x != 0ull;
                }
                if (!__any_sync(0xffffffffu, diff)) return;
            }
        }
        pos = (pos + 1) & ar.slot_mask;
    }
    if (lane == 0) atomicOr(ar.counters + kStatus, kStHashFull);
}

// Vertex of planes p, q and the face plane f (Eq. 11 with biases) by Cramer's rule with cross
// products; optionally the infinity norm of the inverse system matrix.
template <class R>
__device__ __forceinline__ bool solve3(const R *p, const R *q, const R *f, R *v, R *inv_norm)
{
    const R c0x = q[1] * f[2] - q[2] * f[1], c0y = q[2] * f[0] - q[0] * f[2], c0z = q[0] * f[1] - q[1] * f[0];
    const R c1x = f[1] * p[2] - f[2] * p[1], c1y = f[2] * p[0] - f[0] * p[2], c1z = f[0] * p[1] - f[1] * p[0];
    const R c2x = p[1] * q[2] - p[2] * q[1], c2y = p[2] * q[0] - p[0] * q[2], c2z = p[0] * q[1] - p[1] * q[0];
    const R det = p[0] * c0x + p[1] * c0y + p[2] * c0z;
    if (det == R(0)) return false;
    const R inv = R(-1) / det;
    v[0] = (p[3] * c0x + q[3] * c1x + f[3] * c2x) * inv;
    v[1] = (p[3] * c0y + q[3] * c1y + f[3] * c2y) * inv;
    v[2] = (p[3] * c0z + q[3] * c1z + f[3] * c2z) * inv;
    if (inv_norm) {
        const R ax = fabs(c0x) + fabs(c1x) + fabs(c2x), ay = fabs(c0y) + fabs(c1y) + fabs(c2y),
                az = fabs(c0z) + fabs(c1z) + fabs(c2z);
        *inv_norm = fmax(ax, fmax(ay, az)) * fabs(inv);
    }
    return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}

}  // namespace am
