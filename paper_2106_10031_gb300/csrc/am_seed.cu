// am_seed.cu -- trigger cells by dichotomy along rays (Alg. 1 step 2; Sec. 4.3.2), with the
// sphere-tracing walk (Sec. 4.3.1) and the random-pair sampling (Sec. 4.3.2) in front of it.
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
    (void)max_w;
    const int words = (max_n + 31) / 32;
    return max_n * (int)sizeof(double) + 3 * words * (int)sizeof(unsigned) + 16 + 64 * (int)sizeof(double);
}

// Forward pass at x: F (returned to every thread) and the pattern bits in `bits`.  H holds every
// hidden layer's output (N values, layer l at row0[l]), which the residual shortcuts read.
__device__ double seed_forward(const NetDev &net, const double *x, double *H, unsigned *bits, double *red)
{
    const int tid = threadIdx.x, T = blockDim.x;
    for (int w = tid; w < (net.N + 31) / 32; w += T) bits[w] = 0u;
    __syncthreads();
    for (int l = 1; l <= net.L; ++l) {
        const int nl = net.width[l], np = l > 1 ? net.width[l - 1] : 0, rl = net.row0[l];
        const double *Cl = net.Cl[l], *AT = net.AT[l];
        const double *hp = l > 1 ? H + net.row0[l - 1] : nullptr;
        const int src = net.sc_src[l];
        const double *hs = src > 0 ? H + net.row0[src] : nullptr, *S = net.sc_S[l];
        const int ns = src > 0 ? net.width[src] : 0;
        for (int k = tid; k < nl; k += T) {
            double a = Cl[k * 4 + 0] * x[0] + Cl[k * 4 + 1] * x[1] + Cl[k * 4 + 2] * x[2] + Cl[k * 4 + 3];
            for (int j = 0; j < np; ++j) {
                const double hj = hp[j];
                if (hj != 0.0) a += AT[(size_t)j * nl + k] * hj;
            }
            if (hs) {                                          // the residual shortcut S_l h_src
                if (S) for (int j = 0; j < ns; ++j) a += S[(size_t)k * ns + j] * hs[j];
                else a += hs[k];
            }
            H[rl + k] = a > 0.0 ? a : net.slope * a;         // ReLU, or leaky with slope != 0
            if (a > 0.0) atomicOr(bits + ((rl + k) >> 5), 1u << ((rl + k) & 31));
        }
        __syncthreads();
    }
    const double *hL = H + net.row0[net.L];
    const int nL = net.width[net.L];
    if (net.M >= 2) {
        // final max pooling (Sec. 5.2): F = max_i F_i, the pooled index j = the first maximum,
        // as its one-hot key bit n_units + j
        double F = 0.0;
        int j = 0;
        for (int i = 0; i < net.M; ++i) {
            const double *wh = net.w_heads + (size_t)i * nL;
            double f = 0.0;
            for (int k = tid; k < nL; k += T) f += wh[k] * hL[k];
            f = warp_sum(f);
            if ((tid & 31) == 0) red[tid >> 5] = f;
            __syncthreads();
            double Fi = net.b_heads[i];
            for (int w = 0; w < T / 32; ++w) Fi += red[w];
            __syncthreads();
            if (i == 0 || Fi > F) { F = Fi; j = i; }
        }
        if (tid == 0) atomicOr(bits + ((net.n_units + j) >> 5), 1u << ((net.n_units + j) & 31));
        __syncthreads();
        return F;
    }
    double f = 0.0;
    for (int k = tid; k < nL; k += T) f += net.w_out[k] * hL[k];
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
    double *H = (double *)smem;
    unsigned *blo = (unsigned *)(H + a.max_n), *bhi = blo + (a.max_n + 31) / 32, *bm = bhi + (a.max_n + 31) / 32;
    double *red = (double *)(((uintptr_t)(bm + (a.max_n + 31) / 32) + 15) & ~(uintptr_t)15);
    const int ray = blockIdx.x, tid = threadIdx.x;
    const double o[3] = {a.origins[ray * 3], a.origins[ray * 3 + 1], a.origins[ray * 3 + 2]};
    const double d[3] = {a.dirs[ray * 3], a.dirs[ray * 3 + 1], a.dirs[ray * 3 + 2]};
    double x[3];

    double tlo = 0.0, thi = a.R;
    for (int c = 0; c < 3; ++c) x[c] = o[c];
    double flo = seed_forward(net, x, H, blo, red);
    for (int c = 0; c < 3; ++c) x[c] = o[c] + a.R * d[c];
    double fhi = seed_forward(net, x, H, bhi, red);
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
        const double fm = seed_forward(net, x, H, bm, red);
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
    ar.parent[id] = -1;
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

// ---- customised triggers (Sec. 4.3)

// grad F at the point whose pattern the last seed_forward left in `bits`, by backpropagation
// through the units: E[r] = dF/dh_r accumulates from every layer that reads unit r (the next
// layer through W_{l+1}^T, and a residual shortcut through S_q^T), then D_r = g'(a_r) E[r] = dF/da_r
// with g' = 1 on active units and the slope (0 for a ReLU) on the others, and
// grad F = sum_l Cl_l[:, 0:3]^T D_l (the layers fed by x, shortcuts from x included).
// E: N doubles (overwrites the forward pass's H); red: 64 doubles.  Every thread returns g.
__device__ void seed_grad(const NetDev &net, const unsigned *bits, double *E, double *red, double g[3])
{
    const int tid = threadIdx.x, T = blockDim.x;
    double gx = 0.0, gy = 0.0, gz = 0.0;
    const int rL = net.row0[net.L], nU = net.M >= 2 ? net.n_units : net.N;
    const double *wo = net.w_out;                   // a pooled net: the head of the pooled index
    if (net.M >= 2)
        for (int i = 0; i < net.M; ++i)
            if ((bits[(nU + i) >> 5] >> ((nU + i) & 31)) & 1u) { wo = net.w_heads + (size_t)i * net.width[net.L]; break; }
    for (int r = tid; r < nU; r += T) E[r] = r >= rL ? wo[r - rL] : 0.0;
    __syncthreads();
    for (int l = net.L; l >= 1; --l) {
        const int nl = net.width[l], rl = net.row0[l];
        const double *Cl = net.Cl[l];
        for (int k = tid; k < nl; k += T) {
            const double gp = (bits[(rl + k) >> 5] >> ((rl + k) & 31)) & 1u ? 1.0 : net.slope;
            const double dk = gp * E[rl + k];
            E[rl + k] = dk;
            gx += Cl[k * 4 + 0] * dk;
            gy += Cl[k * 4 + 1] * dk;
            gz += Cl[k * 4 + 2] * dk;
        }
        __syncthreads();
        if (l > 1) {
            const int np = net.width[l - 1], rp = net.row0[l - 1];
            const double *AT = net.AT[l];
            for (int j = tid; j < np; j += T) {
                double acc = 0.0;
                for (int k = 0; k < nl; ++k) acc += AT[(size_t)j * nl + k] * E[rl + k];
                E[rp + j] += acc;
            }
            __syncthreads();
        }
        const int src = net.sc_src[l];
        if (src > 0) {
            const int ns = net.width[src], rs = net.row0[src];
            const double *S = net.sc_S[l];
            for (int j = tid; j < ns; j += T) {
                double acc = 0.0;
                if (S) for (int k = 0; k < nl; ++k) acc += S[(size_t)k * ns + j] * E[rl + k];
                else acc = E[rl + j];
                E[rs + j] += acc;
            }
            __syncthreads();
        }
    }
    gx = warp_sum(gx); gy = warp_sum(gy); gz = warp_sum(gz);
    if ((tid & 31) == 0) { red[(tid >> 5) * 3 + 0] = gx; red[(tid >> 5) * 3 + 1] = gy; red[(tid >> 5) * 3 + 2] = gz; }
    __syncthreads();
    g[0] = g[1] = g[2] = 0.0;
    for (int w = 0; w < T / 32; ++w) { g[0] += red[w * 3]; g[1] += red[w * 3 + 1]; g[2] += red[w * 3 + 2]; }
    __syncthreads();
}

// Sphere tracing (Sec. 4.3.1), one block per start point: x <- x - eta F(x) grad F(x) until
// |F| <= eps or max_steps steps, then the bracket along the unit gradient n through the last
// point: o = x - h n, d = 2h n with h = 2|F|/|grad F| + pad, bisected over t in [0, 1] by
// seed_kernel.  A cell with grad F = 0 leaves d = 0, which seed_kernel reports as a ray
// without a sign change.
__global__ void __launch_bounds__(kSeedThreads) trace_kernel(TraceArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const NetDev &net = a.nets[a.net];
    double *H = (double *)smem;
    unsigned *bits = (unsigned *)(H + a.max_n);
    double *red = (double *)(((uintptr_t)(bits + 3 * ((a.max_n + 31) / 32)) + 15) & ~(uintptr_t)15);
    const int i = blockIdx.x, tid = threadIdx.x;
    double x[3] = {a.starts[i * 3], a.starts[i * 3 + 1], a.starts[i * 3 + 2]};
    double F = 0.0, g[3] = {0.0, 0.0, 0.0};
    bool flat = false;
    for (int t = 0;; ++t) {
        F = seed_forward(net, x, H, bits, red);
        seed_grad(net, bits, H, red, g);
        if (fabs(F) <= a.eps || t >= a.max_steps) break;
        if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) { flat = true; break; }
        for (int c = 0; c < 3; ++c) x[c] = x[c] - a.eta * F * g[c];
    }
    if (tid == 0) {
        if (flat) {
            for (int c = 0; c < 3; ++c) { a.origins[i * 3 + c] = x[c]; a.dirs[i * 3 + c] = 0.0; }
        } else {
            const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            const double h = 2.0 * fabs(F) / gn + a.pad;
            for (int c = 0; c < 3; ++c) {
                const double n = g[c] / gn;
                a.origins[i * 3 + c] = x[c] - h * n;
                a.dirs[i * 3 + c] = (2.0 * h) * n;
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// The same forward pass in double-float arithmetic, kDfPts points per block, for nets without
// hidden shortcuts, pooling or leaky units: the pairs (hi, lo) of FP32 words carry about 44 bits
// (the product of two pairs split exactly by an FMA, sums by TwoSum), so F and the pattern bits
// agree with an FP64 evaluation wherever they are not within ~1e-12 of zero.  Each weight pair
// is read once per block for all its points, and the arithmetic runs on the FP32 pipes (this
// part's FP64 pipe is 1/64 of them).

constexpr int kDfPts = 8;                  // points per block
constexpr int kDfW = kSeedThreads / 32;

__host__ __device__ inline int df_seed_smem_bytes(int max_n, int max_w)
{
    const int words = (max_n + 31) / 32;
    return 2 * max_w * 2 * kDfPts * (int)sizeof(float)           // two layers' outputs: [j][hi x 8 | lo x 8]
           + 3 * kDfPts * words * (int)sizeof(unsigned)          // patterns: the bracket's ends, the midpoint
           + kDfPts * 8 * (int)sizeof(float)                     // the points as pairs
           + kDfPts * kDfW * 2 * (int)sizeof(float)              // partial sums of F
           + kDfPts * (int)sizeof(double) + 64;
}

struct DfSm {
    float *h[2];                // layer outputs, element (j, p): hi at [16 j + p], lo at [16 j + 8 + p]
    unsigned *blo, *bhi, *bm;   // patterns, point p at [p words]
    float *xp;                  // point p: [xh, yh, zh, xl, yl, zl] at [8 p]
    float *red;
    double *F;
};

__device__ inline DfSm df_carve(unsigned char *base, int max_n, int max_w)
{
    const int words = (max_n + 31) / 32;
    DfSm s;
    float *f = reinterpret_cast<float *>(base);
    s.h[0] = f;
    s.h[1] = f + 16 * max_w;
    unsigned *u = reinterpret_cast<unsigned *>(f + 32 * max_w);
    s.blo = u;
    s.bhi = u + kDfPts * words;
    s.bm = u + 2 * kDfPts * words;
    s.xp = reinterpret_cast<float *>(u + 3 * kDfPts * words);
    s.red = s.xp + 8 * kDfPts;
    s.F = reinterpret_cast<double *>(((uintptr_t)(s.red + 2 * kDfW * kDfPts) + 15) & ~(uintptr_t)15);
    return s;
}

// (sh, sl) += (ah + al)(zh + zl): TwoProd of the hi words by FMA, the cross terms into the
// error, TwoSum into the sum
__device__ __forceinline__ void dfs_fma(float &sh, float &sl, float ah, float al, float zh, float zl)
{
    const float p = __fmul_rn(ah, zh);
    float pe = __fmaf_rn(ah, zh, -p);
    pe = __fmaf_rn(ah, zl, pe);
    pe = __fmaf_rn(al, zh, pe);
    const float t = __fadd_rn(sh, p);
    const float bp = __fsub_rn(t, sh);
    const float te = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(te, pe));
}

__device__ __forceinline__ void dfs_add(float &sh, float &sl, float bh, float bl)
{
    const float t = __fadd_rn(sh, bh);
    const float bp = __fsub_rn(t, sh);
    const float te = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(bh, bp));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(te, bl));
}

// point p of the block at x (thread p): its coordinates as pairs
__device__ __forceinline__ void df_set_point(const DfSm &s, int p, const double *x)
{
    for (int c = 0; c < 3; ++c) {
        const float h = (float)x[c];
        s.xp[8 * p + c] = h;
        s.xp[8 * p + 3 + c] = (float)(x[c] - (double)h);
    }
}

// F at the block's first NP points (s.xp; the caller sets each of them, unused ones anywhere
// finite) into s.F, and their patterns (Def. 2) into bits[p words].  Every thread calls it.
// NP is 8, 4, 2 or 1: a dichotomy whose other rays are done evaluates only what is left.
template <int NP>
__device__ void df_forward_batch(const NetDev &net, const DfSm &s, unsigned *bits)
{
    static_assert(NP == 1 || NP == 2 || NP == 4 || NP == 8, "points per pass");
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, wid = tid >> 5;
    const int words = (net.N + 31) / 32;
    for (int w = tid; w < NP * words; w += T) bits[w] = 0u;
    __syncthreads();
    for (int l = 1; l <= net.L; ++l) {
        const int nl = net.width[l], np = l > 1 ? net.width[l - 1] : 0, rl = net.row0[l];
        const float *Ch = net.Clhi[l], *Cc = net.Cllo[l];
        const float *Ah = net.AThi[l], *Al = net.ATlo[l];
        const float *ph = s.h[(l - 1) & 1];
        float *out = s.h[l & 1];
        for (int k = tid; k < nl; k += T) {
            float sh[NP], sl[NP];
            const float bh = Ch[4 * k + 3], bl = Cc[4 * k + 3];
#pragma unroll
            for (int p = 0; p < NP; ++p) { sh[p] = bh; sl[p] = bl; }
            for (int c = 0; c < 3; ++c) {                // the input columns (layer 1, and skip layers)
                const float wh = Ch[4 * k + c], wl = Cc[4 * k + c];
                if (wh == 0.0f && wl == 0.0f) continue;
#pragma unroll
                for (int p = 0; p < NP; ++p) dfs_fma(sh[p], sl[p], wh, wl, s.xp[8 * p + c], s.xp[8 * p + 3 + c]);
            }
            for (int j = 0; j < np; ++j) {
                const float ah = __ldg(Ah + (size_t)j * nl + k), al = __ldg(Al + (size_t)j * nl + k);
                float zh[NP], zl[NP];
                if constexpr (NP >= 4) {
                    const float4 *hj = reinterpret_cast<const float4 *>(ph + 16 * j);
#pragma unroll
                    for (int g = 0; g < NP / 4; ++g) {
                        const float4 h4 = hj[g], l4 = hj[2 + g];
                        zh[4 * g] = h4.x; zh[4 * g + 1] = h4.y; zh[4 * g + 2] = h4.z; zh[4 * g + 3] = h4.w;
                        zl[4 * g] = l4.x; zl[4 * g + 1] = l4.y; zl[4 * g + 2] = l4.z; zl[4 * g + 3] = l4.w;
                    }
                } else {
#pragma unroll
                    for (int p = 0; p < NP; ++p) { zh[p] = ph[16 * j + p]; zl[p] = ph[16 * j + 8 + p]; }
                }
#pragma unroll
                for (int p = 0; p < NP; ++p) dfs_fma(sh[p], sl[p], ah, al, zh[p], zl[p]);
            }
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const float t = __fadd_rn(sh[p], sl[p]);       // renormalise: sign(pair) = sign(hi)
                const float lo = __fsub_rn(sl[p], __fsub_rn(t, sh[p]));
                const bool act = t > 0.0f;
                out[16 * k + p] = act ? t : 0.0f;
                out[16 * k + 8 + p] = act ? lo : 0.0f;
                if (act) atomicOr(bits + p * words + ((rl + k) >> 5), 1u << ((rl + k) & 31));
            }
        }
        __syncthreads();
    }
    const int nL = net.width[net.L];
    const float *hL = s.h[net.L & 1];
    float fh[NP], fl[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) { fh[p] = 0.0f; fl[p] = 0.0f; }
    for (int k = tid; k < nL; k += T) {
        const float wh = net.w_out_hi[k], wl = net.w_out_lo[k];
#pragma unroll
        for (int p = 0; p < NP; ++p) dfs_fma(fh[p], fl[p], wh, wl, hL[16 * k + p], hL[16 * k + 8 + p]);
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, fh[p], o), ol = __shfl_xor_sync(0xffffffffu, fl[p], o);
            dfs_add(fh[p], fl[p], oh, ol);
        }
        if (lane == 0) { s.red[2 * (p * kDfW + wid)] = fh[p]; s.red[2 * (p * kDfW + wid) + 1] = fl[p]; }
    }
    __syncthreads();
    if (tid < NP) {
        double F = net.b_out;
        for (int w = 0; w < T / 32; ++w) F += (double)s.red[2 * (tid * kDfW + w)] + (double)s.red[2 * (tid * kDfW + w) + 1];
        s.F[tid] = F;
    }
    __syncthreads();
}

// the forward pass of the first n (1..8) points, in the smallest batch that holds them
__device__ void df_forward_n(const NetDev &net, const DfSm &s, unsigned *bits, int n)
{
    if (n > 4) df_forward_batch<8>(net, s, bits);
    else if (n > 2) df_forward_batch<4>(net, s, bits);
    else if (n > 1) df_forward_batch<2>(net, s, bits);
    else df_forward_batch<1>(net, s, bits);
}

// F at every sample point (random-pair trigger, Sec. 4.3.2), kDfPts points per block
__global__ void __launch_bounds__(kSeedThreads) sample_eval_df_kernel(PairArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const NetDev &net = a.nets[a.net];
    const DfSm s = df_carve(smem, a.max_n, a.max_w);
    const int i0 = blockIdx.x * kDfPts, P = min(kDfPts, a.n_points - i0);
    if (threadIdx.x < kDfPts) {
        const int i = i0 + (threadIdx.x < P ? threadIdx.x : 0);
        const double x[3] = {a.points[3 * i], a.points[3 * i + 1], a.points[3 * i + 2]};
        df_set_point(s, threadIdx.x, x);
    }
    __syncthreads();
    df_forward_n(net, s, s.bm, P);
    if (threadIdx.x < P) a.F[i0 + threadIdx.x] = s.F[threadIdx.x];
}

// The dichotomy of seed_kernel for kDfPts rays per block, in double-float: one batched forward
// pass per halving step of the block's rays that still bracket more than one cell, packed into
// the first slots so that a step with fewer rays left evaluates fewer points.
__global__ void __launch_bounds__(kSeedThreads) seed_df_kernel(SeedArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double tlo[kDfPts], thi[kDfPts], flo[kDfPts], fhi[kDfPts], tm[kDfPts];
    __shared__ int rc[kDfPts], act[kDfPts], side[kDfPts], slot_ray[kDfPts], n_act;
    const NetDev &net = a.nets[a.net];
    const DfSm s = df_carve(smem, a.max_n, a.max_w);
    const int tid = threadIdx.x, words = (net.N + 31) / 32;
    const int r0 = blockIdx.x * kDfPts, P = min(kDfPts, a.n_rays - r0);
    auto point = [&](int q, int p, double t) {          // slot q: ray p's point at t (rays past P: ray 0)
        const int r = r0 + (p < P ? p : 0);
        const double x[3] = {a.origins[3 * r] + t * a.dirs[3 * r], a.origins[3 * r + 1] + t * a.dirs[3 * r + 1],
                             a.origins[3 * r + 2] + t * a.dirs[3 * r + 2]};
        df_set_point(s, q, x);
    };
    if (tid < kDfPts) { tlo[tid] = 0.0; thi[tid] = a.R; point(tid, tid, 0.0); }
    __syncthreads();
    df_forward_n(net, s, s.blo, P);
    if (tid < kDfPts) { flo[tid] = s.F[tid]; point(tid, tid, a.R); }
    __syncthreads();
    df_forward_n(net, s, s.bhi, P);
    if (tid < kDfPts) {
        fhi[tid] = s.F[tid];
        const double f0 = flo[tid], f1 = fhi[tid];
        rc[tid] = tid >= P ? 0 : ((f0 < 0.0 && f1 > 0.0) || (f0 > 0.0 && f1 < 0.0)) ? 1 : -4;
    }
    __syncthreads();
    for (int it = 0;; ++it) {
        if (tid < kDfPts) {
            int diff = 0;
            if (rc[tid] == 1)
                for (int w = 0; w < words; ++w) diff |= s.blo[tid * words + w] != s.bhi[tid * words + w];
            act[tid] = diff;
            side[tid] = 0;
        }
        __syncthreads();
        if (tid == 0) {
            int q = 0;
            for (int p = 0; p < kDfPts; ++p)
                if (act[p]) slot_ray[q++] = p;
            n_act = q;
        }
        __syncthreads();
        const int nact = n_act;
        if (nact == 0) break;
        if (it >= a.max_halvings) {
            if (tid < kDfPts && act[tid]) rc[tid] = -5;
            break;
        }
        if (tid < nact) {
            const int p = slot_ray[tid];
            tm[p] = 0.5 * (tlo[p] + thi[p]);
            point(tid, p, tm[p]);
        }
        __syncthreads();
        df_forward_n(net, s, s.bm, nact);
        if (tid < nact) {
            const int p = slot_ray[tid];
            const double fm = s.F[tid];
            if ((fm < 0.0) == (flo[p] < 0.0) && fm != 0.0) { tlo[p] = tm[p]; flo[p] = fm; side[p] = 1; }
            else { thi[p] = tm[p]; fhi[p] = fm; side[p] = 2; }
        }
        __syncthreads();
        for (int q = tid; q < nact * words; q += blockDim.x) {
            const int slot = q / words, w = q - slot * words, p = slot_ray[slot];
            if (side[p] == 1) s.blo[p * words + w] = s.bm[q];
            else if (side[p] == 2) s.bhi[p * words + w] = s.bm[q];
        }
        __syncthreads();
    }
    __syncthreads();
    for (int p = 0; p < P; ++p) {
        const int ray = r0 + p;
        if (rc[p] == 1) {
            const double ts = tlo[p] + flo[p] / (flo[p] - fhi[p]) * (thi[p] - tlo[p]);
            if (tid < 3) a.seed_x[ray * 3 + tid] = a.origins[ray * 3 + tid] + ts * a.dirs[ray * 3 + tid];
            for (int w = tid; w < a.ar.kw; w += blockDim.x) {
                const unsigned lo = 2 * w < words ? s.blo[p * words + 2 * w] : 0u;
                const unsigned hi = 2 * w + 1 < words ? s.blo[p * words + 2 * w + 1] : 0u;
                a.seed_keys[(size_t)ray * a.ar.kw + w] = (unsigned long long)lo | ((unsigned long long)hi << 32);
            }
        } else if (tid == 0) {
            atomicOr(a.ar.counters + kStatus, rc[p] == -4 ? kStSeedNoSign : kStSeedNoCell);
        }
        if (tid == 0) a.seed_ok[ray] = rc[p];
    }
}

// F at every sample point (random-pair trigger, Sec. 4.3.2), one block per point.
__global__ void __launch_bounds__(kSeedThreads) sample_eval_kernel(PairArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const NetDev &net = a.nets[a.net];
    double *H = (double *)smem;
    unsigned *bits = (unsigned *)(H + a.max_n);
    double *red = (double *)(((uintptr_t)(bits + 3 * ((a.max_n + 31) / 32)) + 15) & ~(uintptr_t)15);
    const int i = blockIdx.x;
    const double x[3] = {a.points[i * 3], a.points[i * 3 + 1], a.points[i * 3 + 2]};
    const double F = seed_forward(net, x, H, bits, red);
    if (threadIdx.x == 0) a.F[i] = F;
}

// Pair the r-th sample with F < 0 and the r-th sample with F > 0 (sample order) for r below
// min(#neg, #pos, max_pairs) and write segment r: origin x-, direction x+ - x- (t in [0, 1]).
// One block of kPairThreads threads walks the samples in chunks; ranks come from a block
// scan of ballot counts.
constexpr int kPairThreads = 1024;
__global__ void __launch_bounds__(kPairThreads) pair_build_kernel(PairArgs a)
{
    __shared__ int wneg[kPairThreads / 32], wpos[kPairThreads / 32];
    __shared__ int base[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) base[0] = base[1] = 0;
    __syncthreads();
    for (int c0 = 0; c0 < a.n_points; c0 += kPairThreads) {
        if (base[0] >= a.max_pairs && base[1] >= a.max_pairs) break;   // block-uniform
        const int i = c0 + tid;
        const double f = i < a.n_points ? a.F[i] : 0.0;
        const bool neg = i < a.n_points && f < 0.0, pos = i < a.n_points && f > 0.0;
        const unsigned bn = __ballot_sync(0xffffffffu, neg), bp = __ballot_sync(0xffffffffu, pos);
        if (lane == 0) { wneg[warp] = __popc(bn); wpos[warp] = __popc(bp); }
        __syncthreads();
        int rn = base[0] + __popc(bn & ((1u << lane) - 1u)), rp = base[1] + __popc(bp & ((1u << lane) - 1u));
        for (int w = 0; w < warp; ++w) { rn += wneg[w]; rp += wpos[w]; }
        if (neg && rn < a.max_pairs) a.neg_idx[rn] = i;
        if (pos && rp < a.max_pairs) a.pos_idx[rp] = i;
        __syncthreads();
        if (tid == 0) {
            int tn = 0, tp = 0;
            for (int w = 0; w < kPairThreads / 32; ++w) { tn += wneg[w]; tp += wpos[w]; }
            base[0] += tn; base[1] += tp;
        }
        __syncthreads();
    }
    const int n_pairs = min(min(base[0], base[1]), a.max_pairs);
    __syncthreads();   // every neg_idx / pos_idx write of the loop is visible below
    for (int r = tid; r < n_pairs; r += kPairThreads) {
        const int in = a.neg_idx[r], ip = a.pos_idx[r];
        for (int c = 0; c < 3; ++c) {
            const double xm = a.points[in * 3 + c];
            a.origins[r * 3 + c] = xm;
            a.dirs[r * 3 + c] = a.points[ip * 3 + c] - xm;
        }
    }
    if (tid == 0) *a.n_pairs = n_pairs;
}

cudaError_t prepare_seed_kernels(int max_n, int max_w)
{
    const int bytes = seed_smem_bytes(max_n, max_w);
    cudaError_t e = cudaFuncSetAttribute(seed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(trace_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sample_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    const int dbytes = df_seed_smem_bytes(max_n, max_w);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sample_eval_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dbytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(seed_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dbytes);
    return e;
}

void launch_trace(const TraceArgs &a, cudaStream_t st)
{
    trace_kernel<<<a.n, kSeedThreads, seed_smem_bytes(a.max_n, a.max_w), st>>>(a);
}

void launch_pairs(const PairArgs &a, cudaStream_t st)
{
    if (a.df)
        sample_eval_df_kernel<<<(a.n_points + kDfPts - 1) / kDfPts, kSeedThreads, df_seed_smem_bytes(a.max_n, a.max_w),
                                st>>>(a);
    else
        sample_eval_kernel<<<a.n_points, kSeedThreads, seed_smem_bytes(a.max_n, a.max_w), st>>>(a);
    pair_build_kernel<<<1, kPairThreads, 0, st>>>(a);
}

void launch_seed(const SeedArgs &a, cudaStream_t st)
{
    if (a.df)
        seed_df_kernel<<<(a.n_rays + kDfPts - 1) / kDfPts, kSeedThreads, df_seed_smem_bytes(a.max_n, a.max_w), st>>>(a);
    else
        seed_kernel<<<a.n_rays, kSeedThreads, seed_smem_bytes(a.max_n, a.max_w), st>>>(a);
    seed_insert_kernel<<<(a.n_rays + 127) / 128, 128, 0, st>>>(a);
}

}  // namespace am
