// am_seed.cu -- trigger cells by dichotomy along rays (Alg. 1 step 2; Sec. 4.3.2).
//
// One thread block per ray.  F and the state pattern (Def. 2) come from a block-parallel
// FP64 forward pass (Eq. 1).  The bracket [t_lo, t_hi] keeps F of opposite signs at its
// ends and is halved until both ends share one activation pattern; inside that cell F is
// affine along the ray, so the root is t* = t_lo + F_lo / (F_lo - F_hi) (t_hi - t_lo).
// A second kernel pushes each new seed cell into the active set (hash table + arena).
#include "am_block.cuh"
#include "am_kernels.h"

namespace am {

constexpr int kSeedThreads = 256;

__host__ __device__ inline int seed_smem_bytes(int max_n, int max_w)
{
    const int words = (max_n + 31) / 32;
    return 2 * max_w * (int)sizeof(double) + 3 * words * (int)sizeof(unsigned) + 16 + 64 * (int)sizeof(double);
}

// Forward pass at x: F (returned to every thread) and the pattern bits in `bits`.
__device__ double seed_forward(const NetDev &net, const double *x, double *h0, double *h1, unsigned *bits,
                               double *red)
{
    const int tid = threadIdx.x, T = blockDim.x;
    for (int w = tid; w < (net.N + 31) / 32; w += T) bits[w] = 0u;
    __syncthreads();
    double *hp = h0, *hn = h1;
    for (int l = 1; l <= net.L; ++l) {
        const int nl = net.width[l], np = l > 1 ? net.width[l - 1] : 0, rl = net.row0[l];
        const double *Cl = net.Cl[l], *AT = net.AT[l];
        for (int k = tid; k < nl; k += T) {
            double a = Cl[k * 4 + 0] * x[0] + Cl[k * 4 + 1] * x[1] + Cl[k * 4 + 2] * x[2] + Cl[k * 4 + 3];
            for (int j = 0; j < np; ++j) {
                const double hj = hp[j];
                if (hj != 0.0) a += AT[(size_t)j * nl + k] * hj;
            }
            hn[k] = a > 0.0 ? a : 0.0;
            if (a > 0.0) atomicOr(bits + ((rl + k) >> 5), 1u << ((rl + k) & 31));
        }
        __syncthreads();
        double *t = hp; hp = hn; hn = t;
    }
    double f = 0.0;
    for (int k = tid; k < net.width[net.L]; k += T) f += net.w_out[k] * hp[k];
    f = warp_sum(f);
    if ((tid & 31) == 0) red[tid >> 5] = f;
    __syncthreads();
    double F = net.b_out;
    for (int w = 0; w < T / 32; ++w) F += red[w];
    __syncthreads();
    return F;
}

__global__ void __launch_bounds__(kSeedThreads) seed_kernel(SeedArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const NetDev &net = a.nets[a.net];
    const int words = (net.N + 31) / 32;
    double *h0 = (double *)smem, *h1 = h0 + a.max_w;
    unsigned *blo = (unsigned *)(h1 + a.max_w), *bhi = blo + (a.max_n + 31) / 32, *bm = bhi + (a.max_n + 31) / 32;
    double *red = (double *)(((uintptr_t)(bm + (a.max_n + 31) / 32) + 15) & ~(uintptr_t)15);
    const int ray = blockIdx.x, tid = threadIdx.x;
    const double o[3] = {a.origins[ray * 3], a.origins[ray * 3 + 1], a.origins[ray * 3 + 2]};
    const double d[3] = {a.dirs[ray * 3], a.dirs[ray * 3 + 1], a.dirs[ray * 3 + 2]};
    double x[3];

    double tlo = 0.0, thi = a.R;
    for (int c = 0; c < 3; ++c) x[c] = o[c];
    double flo = seed_forward(net, x, h0, h1, blo, red);
    for (int c = 0; c < 3; ++c) x[c] = o[c] + a.R * d[c];
    double fhi = seed_forward(net, x, h0, h1, bhi, red);
    int rc = 1;
    if (!((flo < 0.0 && fhi > 0.0) || (flo > 0.0 && fhi < 0.0))) rc = -4;
    int it = 0;
    while (rc == 1) {
        int diff = 0;
        for (int w = tid; w < words; w += blockDim.x) diff |= (blo[w] != bhi[w]);
        diff = __syncthreads_or(diff);
        if (!diff) break;
        if (it >= a.max_halvings) { rc = -5; break; }
        const double tm = 0.5 * (tlo + thi);
        for (int c = 0; c < 3; ++c) x[c] = o[c] + tm * d[c];
        const double fm = seed_forward(net, x, h0, h1, bm, red);
        if ((fm < 0.0) == (flo < 0.0) && fm != 0.0) {
            tlo = tm; flo = fm;
            for (int w = tid; w < words; w += blockDim.x) blo[w] = bm[w];
        } else {
            thi = tm; fhi = fm;
            for (int w = tid; w < words; w += blockDim.x) bhi[w] = bm[w];
        }
        __syncthreads();
        ++it;
    }
    if (tid == 0) a.seed_ok[ray] = rc;
    if (rc == 1) {
        const double ts = tlo + flo / (flo - fhi) * (thi - tlo);
        if (tid < 3) a.seed_x[ray * 3 + tid] = o[tid] + ts * d[tid];
        for (int w = tid; w < a.ar.kw; w += blockDim.x) {
            const unsigned lo = 2 * w < words ? blo[2 * w] : 0u;
            const unsigned hi = 2 * w + 1 < words ? blo[2 * w + 1] : 0u;
            a.seed_keys[(size_t)ray * a.ar.kw + w] = (unsigned long long)lo | ((unsigned long long)hi << 32);
        }
    } else if (tid == 0) {
        atomicOr(a.ar.counters + kStatus, rc == -4 ? kStSeedNoSign : kStSeedNoCell);
    }
}

// Push the seed cells: allocate an id, write the key, then claim the hash slot with the
// ref (id, no flip).  A ray landing in an already known cell marks its id dead (-2).
__global__ void seed_insert_kernel(SeedArgs a)
{
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= a.n_rays || a.seed_ok[ray] != 1) return;
    const Arena &ar = a.ar;
    const NetDev &net = a.nets[a.net];
    const unsigned long long *k = a.seed_keys + (size_t)ray * ar.kw;
    unsigned long long h = net.salt;
    for (int w = 0; w < ar.kw; ++w) {
        unsigned long long x = k[w];
        while (x) {
            const int b = __ffsll((long long)x) - 1;
            h ^= ar.zob[w * 64 + b];
            x &= x - 1;
        }
    }
    const long long id = (long long)atomicAdd(ar.counters + kNCells, 1ull);
    if (id >= ar.cap) { atomicOr(ar.counters + kStatus, kStCellCap); return; }
    for (int w = 0; w < ar.kw; ++w) ar.keys[id * ar.kw + w] = k[w];
    ar.net[id] = a.net;
    ar.hash[id] = h;
    ar.nverts[id] = -1;
    ar.entry_plane[id] = -1;
    for (int c = 0; c < 3; ++c) ar.entry_pt[id * 3 + c] = (float)a.seed_x[ray * 3 + c];
    __threadfence();
    const unsigned long long mine = slot_make(h, (unsigned long long)id, kNoFlip);
    unsigned long long pos = h & ar.slot_mask;
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        unsigned long long cur = atomicCAS(ar.slots + pos, 0ull, mine);
        if (cur == 0ull) {
            atomicAdd(a.n_new, 1ull);
            atomicExch(ar.ready + id, 1u);
            return;
        }
        if (slot_tag(cur) == hash_tag(h) && __ldcg(ar.net + slot_parent(cur)) == a.net &&
            ref_keys_equal(ar, id, kNoFlip, slot_parent(cur), slot_flip(cur))) {
            ar.nverts[id] = -2;
            atomicExch(ar.ready + id, 1u);
            return;
        }
        pos = (pos + 1) & ar.slot_mask;
    }
    ar.nverts[id] = -2;
    atomicExch(ar.ready + id, 1u);
    atomicOr(ar.counters + kStatus, kStHashFull);
}

cudaError_t prepare_seed_kernels(int max_n, int max_w)
{
    return cudaFuncSetAttribute(seed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                seed_smem_bytes(max_n, max_w));
}

void launch_seed(const SeedArgs &a, cudaStream_t st)
{
    seed_kernel<<<a.n_rays, kSeedThreads, seed_smem_bytes(a.max_n, a.max_w), st>>>(a);
    seed_insert_kernel<<<(a.n_rays + 127) / 128, 128, 0, st>>>(a);
}

}  // namespace am
