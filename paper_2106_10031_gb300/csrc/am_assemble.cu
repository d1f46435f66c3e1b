// am_assemble.cu -- mesh assembly (a8): Z = {V, {P}} from the solved cells.
//
// Faces are grouped by net (counting sort on the net id), corner offsets come from an
// exclusive scan of the face sizes, and vertices are deduplicated by their combinatorial
// key (i, j, s with bits i and j cleared; i < j the planes meeting there) in a hash table,
// so the faces meeting at a vertex share one index without comparing coordinates.
#include "am_block.cuh"
#include "am_kernels.h"

namespace am {

constexpr int kAsmThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int32_t kWinBit = 1 << 30;
constexpr int32_t kUnset = -1;

__global__ void asm_count_kernel(AsmArgs a)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < a.n_cells; c += (int64_t)gridDim.x * blockDim.x)
        if (a.ar.nverts[c] > 0) atomicAdd(a.face_count + a.ar.net[c], 1ull);
}

__global__ void asm_scatter_kernel(AsmArgs a)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < a.n_cells; c += (int64_t)gridDim.x * blockDim.x) {
        const int nv = a.ar.nverts[c];
        if (nv <= 0) continue;
        const int net = a.ar.net[c];
        const unsigned long long pos = a.face_base[net] + atomicAdd(a.face_fill + net, 1ull);
        a.perm[pos] = (int32_t)c;
        a.corner_off[pos] = nv;
    }
}

// ---- exclusive scan of int64 (three passes; up to kScanThreads*kScanPer blocks)
__global__ void scan_blocks_kernel(int64_t *v, int64_t n, int64_t *tops)
{
    __shared__ int64_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanThreads * kScanPer + threadIdx.x * kScanPer;
    int64_t x[kScanPer], s = 0;
    for (int i = 0; i < kScanPer; ++i) { x[i] = base + i < n ? v[base + i] : 0; s += x[i]; }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t t = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    int64_t run = (wid ? ws[wid - 1] : 0) + inc - s;
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < n) v[base + i] = run;
        run += x[i];
    }
    if (threadIdx.x == kScanThreads - 1) tops[blockIdx.x] = (wid ? ws[wid - 1] : 0) + inc;
}

__global__ void scan_add_kernel(int64_t *v, int64_t n, const int64_t *tops_excl)
{
    const int64_t add = tops_excl[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kScanThreads * kScanPer;
    for (int i = threadIdx.x; i < kScanThreads * kScanPer; i += blockDim.x)
        if (base + i < n) v[base + i] += add;
}

// in-place exclusive scan of v[0..n), writes the total to v[n].  tmp: >= 2 * blocks + 4 (the
// block totals, scanned the same way, recursively, while they span more than one block).
static cudaError_t exclusive_scan(int64_t *v, int64_t n, int64_t *tmp, int64_t tmp_len, cudaStream_t st)
{
    const int64_t per = (int64_t)kScanThreads * kScanPer;
    if (n == 0) return cudaMemsetAsync(v, 0, sizeof(int64_t), st);
    const int64_t blocks = (n + per - 1) / per;
    if (blocks + 2 > tmp_len) return cudaErrorInvalidValue;
    scan_blocks_kernel<<<(unsigned)blocks, kScanThreads, 0, st>>>(v, n, tmp);   // block totals to tmp
    if (blocks == 1) return cudaMemcpyAsync(v + n, tmp, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    cudaError_t e = exclusive_scan(tmp, blocks, tmp + blocks + 1, tmp_len - blocks - 1, st);
    if (e != cudaSuccess) return e;
    scan_add_kernel<<<(unsigned)blocks, 256, 0, st>>>(v, n, tmp);
    return cudaMemcpyAsync(v + n, tmp + blocks, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
}

// ---- vertex keys
constexpr int kPairCode = 1 << 20;      // codes of pooling planes and of their triple points
constexpr int kTripleCode = 1 << 24;

// The two planes meeting at corner j of a cell's face (edges j - 1 and j), as codes that every
// face sharing the vertex gives it alike, lo <= hi.  Unit and box planes are their ids.  On a
// max-pooled net (Sec. 5.2) the pooling plane between heads i and j, which the cell of pooled
// index j names N_units + i and the cell of index i names N_units + j, is the pair {i, j}; a
// vertex on two pooling planes is the triple of their heads.  *pool: the vertex lies on a
// pooling plane, so its key leaves out the pooled index.
__device__ __forceinline__ void corner_planes(const Arena &ar, const NetDev &net, int32_t cell, int nv, int j, int *lo,
                                              int *hi, bool *pool)
{
    int a = ar.edges[(int64_t)cell * ar.maxv + (j + nv - 1) % nv];
    int b = ar.edges[(int64_t)cell * ar.maxv + j];
    *pool = false;
    if (net.M >= 2) {
        const bool pa = a >= net.n_units && a < net.N, pb = b >= net.n_units && b < net.N;
        if (pa || pb) {
            *pool = true;
            const int own = pooled_index(net, ar.keys + (int64_t)cell * ar.kw);
            if (pa && pb) {
                int t0 = a - net.n_units, t1 = b - net.n_units, t2 = own, t;
                if (t0 > t1) { t = t0; t0 = t1; t1 = t; }
                if (t1 > t2) { t = t1; t1 = t2; t2 = t; }
                if (t0 > t1) { t = t0; t0 = t1; t1 = t; }
                a = b = kTripleCode + ((t0 << 12) | (t1 << 6) | t2);
            } else {
                const int i = (pa ? a : b) - net.n_units;
                const int code = kPairCode + ((min(i, own) << 6) | max(i, own));
                if (pa) a = code;
                else b = code;
            }
        }
    }
    *lo = a < b ? a : b;
    *hi = a < b ? b : a;
}

// the first plane id that is not a unit (a pooled net's pooling planes carry the one-hot index)
__device__ __forceinline__ int unit_planes(const NetDev &net) { return net.M >= 2 ? net.n_units : net.N; }

__device__ __forceinline__ unsigned long long vertex_hash(const Arena &ar, const NetDev &net, int32_t cell, int lo,
                                                          int hi, bool pool)
{
    unsigned long long h = ar.hash[cell];
    const unsigned long long *k = ar.keys + (int64_t)cell * ar.kw;
    const int nU = unit_planes(net);
    if (lo < nU && ((k[lo >> 6] >> (lo & 63)) & 1ull)) h ^= ar.zob[lo];
    if (hi < nU && ((k[hi >> 6] >> (hi & 63)) & 1ull)) h ^= ar.zob[hi];
    if (pool) h ^= ar.zob[net.n_units + pooled_index(net, k)];
    return h ^ splitmix64(((unsigned long long)lo << 20) ^ (unsigned long long)hi ^ 0x5bd1e995ull);
}

__device__ __forceinline__ bool vertex_keys_equal(const Arena &ar, const NetDev &net, int32_t c1, int32_t c2, int lo,
                                                  int hi, bool pool)
{
    const unsigned long long *k1 = ar.keys + (int64_t)c1 * ar.kw, *k2 = ar.keys + (int64_t)c2 * ar.kw;
    const int nU = unit_planes(net);
    for (int w = 0; w < ar.kw; ++w) {
        unsigned long long x = k1[w] ^ k2[w];
        if (lo < nU && (lo >> 6) == w) x &= ~(1ull << (lo & 63));
        if (hi < nU && (hi >> 6) == w) x &= ~(1ull << (hi & 63));
        if (pool) {
            const int a = max(net.n_units - 64 * w, 0), b = min(net.N - 64 * w, 64);
            if (a < b) x &= ~((b >= 64 ? ~0ull : ((1ull << b) - 1ull)) & ~((1ull << a) - 1ull));
        }
        if (x) return false;
    }
    return true;
}

__device__ __forceinline__ unsigned long long vslot_make(unsigned long long h, int64_t face, int corner)
{
    return (1ull << 63) | (((h >> 41) & 0x7FFFFFull) << 40) | (((unsigned long long)face & 0x3FFFFFFFFull) << 6) |
           (unsigned long long)(corner & 63);
}

// find (or claim) the slot of vertex (lo, hi, key of cell) (corner j of face `face`, codes of
// corner_planes); returns the slot value
__device__ unsigned long long vertex_probe(const AsmArgs &a, const NetDev &net, int64_t face, int j, int32_t cell,
                                           int net_id, int lo, int hi, bool pool, bool claim, bool *claimed)
{
    const unsigned long long h = vertex_hash(a.ar, net, cell, lo, hi, pool);
    const unsigned long long mine = vslot_make(h, face, j);
    unsigned long long pos = h & a.vslot_mask;
    *claimed = false;
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        unsigned long long cur = *((volatile unsigned long long *)(a.vslots + pos));
        if (cur == 0ull && claim) {
            cur = atomicCAS(a.vslots + pos, 0ull, mine);
            if (cur == 0ull) { *claimed = true; return mine; }
        }
        if (cur == 0ull) return 0ull;
        if (((cur >> 40) & 0x7FFFFFull) == ((h >> 41) & 0x7FFFFFull)) {
            const int64_t f2 = (int64_t)((cur >> 6) & 0x3FFFFFFFFull);
            const int j2 = (int)(cur & 63);
            const int32_t c2 = a.perm[f2];
            if (a.ar.net[c2] == net_id) {
                int lo2, hi2;
                bool pool2;
                corner_planes(a.ar, net, c2, a.ar.nverts[c2], j2, &lo2, &hi2, &pool2);
                if (lo2 == lo && hi2 == hi && vertex_keys_equal(a.ar, net, cell, c2, lo, hi, pool)) return cur;
            }
        }
        pos = (pos + 1) & a.vslot_mask;
    }
    atomicOr(a.ar.counters + kStatus, kStVertHash);
    return 0ull;
}

__global__ void asm_vertices_kernel(AsmArgs a)
{
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < a.n_faces; f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = a.perm[f];
        const int nv = a.ar.nverts[c], net_id = a.ar.net[c];
        const NetDev &net = a.nets[net_id];
        const int64_t off = a.corner_off[f];
        for (int j = 0; j < nv; ++j) {
            int lo, hi;
            bool pool;
            corner_planes(a.ar, net, c, nv, j, &lo, &hi, &pool);
            bool claimed;
            vertex_probe(a, net, f, j, c, net_id, lo, hi, pool, true, &claimed);
            if (claimed) {
                const int32_t vid = (int32_t)atomicAdd(a.vert_count + net_id, 1ull);
                a.corner_vid[off + j] = vid | kWinBit;
            } else {
                a.corner_vid[off + j] = kUnset;
            }
        }
    }
}

__global__ void asm_lookup_kernel(AsmArgs a)
{
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < a.n_faces; f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = a.perm[f];
        const int nv = a.ar.nverts[c], net_id = a.ar.net[c];
        const NetDev &net = a.nets[net_id];
        const int64_t off = a.corner_off[f];
        for (int j = 0; j < nv; ++j) {
            if (a.corner_vid[off + j] != kUnset) continue;
            int lo, hi;
            bool pool;
            corner_planes(a.ar, net, c, nv, j, &lo, &hi, &pool);
            bool claimed;
            const unsigned long long s = vertex_probe(a, net, f, j, c, net_id, lo, hi, pool, false, &claimed);
            if (s == 0ull) continue;
            const int64_t f2 = (int64_t)((s >> 6) & 0x3FFFFFFFFull);
            const int j2 = (int)(s & 63);
            a.corner_vid[off + j] = a.corner_vid[a.corner_off[f2] + j2] & ~kWinBit;
        }
    }
}

__global__ void asm_write_kernel(AsmArgs a)
{
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < a.n_faces; f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = a.perm[f];
        const int nv = a.ar.nverts[c], net_id = a.ar.net[c];
        const int64_t off = a.corner_off[f];
        for (int j = 0; j < nv; ++j) {
            const int32_t v = a.corner_vid[off + j];
            const int32_t vid = v & ~kWinBit;
            a.out_fv[off + j] = v == kUnset ? -1 : vid;
            a.out_edges[off + j] = a.ar.edges[(int64_t)c * a.ar.maxv + j];
            if (v != kUnset && (v & kWinBit)) {
                const double *p = a.ar.verts + ((int64_t)c * a.ar.maxv + j) * 3;
                double *q = a.out_xyz + (a.vert_base[net_id] + vid) * 3;
                q[0] = p[0]; q[1] = p[1]; q[2] = p[2];
            }
        }
        for (int w = 0; w < a.ar.kw; ++w) a.out_keys[f * a.ar.kw + w] = a.ar.keys[(int64_t)c * a.ar.kw + w];
    }
}

static int grid_for(int64_t n)
{
    int64_t g = (n + kAsmThreads - 1) / kAsmThreads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

void launch_asm_count(const AsmArgs &a, cudaStream_t st) { asm_count_kernel<<<grid_for(a.n_cells), kAsmThreads, 0, st>>>(a); }
void launch_asm_scatter(const AsmArgs &a, cudaStream_t st) { asm_scatter_kernel<<<grid_for(a.n_cells), kAsmThreads, 0, st>>>(a); }
cudaError_t launch_asm_offsets(const AsmArgs &a, int64_t *tmp, int64_t tmp_len, cudaStream_t st)
{
    return exclusive_scan(a.corner_off, a.n_faces, tmp, tmp_len, st);
}
void launch_asm_vertices(const AsmArgs &a, cudaStream_t st) { asm_vertices_kernel<<<grid_for(a.n_faces), kAsmThreads, 0, st>>>(a); }
void launch_asm_lookup(const AsmArgs &a, cudaStream_t st) { asm_lookup_kernel<<<grid_for(a.n_faces), kAsmThreads, 0, st>>>(a); }
void launch_asm_write(const AsmArgs &a, cudaStream_t st) { asm_write_kernel<<<grid_for(a.n_faces), kAsmThreads, 0, st>>>(a); }

// out[i] = in[i] - base for i < n: one net's face offsets relative to its first corner
__global__ void rebase_offsets_kernel(const int64_t *in, int64_t base, int64_t *out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] - base;
}

void launch_rebase_offsets(const int64_t *in, int64_t base, int64_t *out, int64_t n, cudaStream_t st)
{
    if (n > 0) rebase_offsets_kernel<<<grid_for(n), kAsmThreads, 0, st>>>(in, base, out, n);
}

}  // namespace am
