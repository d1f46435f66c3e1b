// am_march.cu -- the march: one thread block solves one analytic cell at a time.
//
// Per cell (Alg. 1 steps 4-11):
//   a2 compose : Z_l = W_l diag(s_{l-1}) Z_{l-1} + C_l (Lemma 1, Cor. 1) over the active
//                neurons of the previous layer, then a_F (Eq. 8);
//   a3 rows    : c_k = (1 - 2 s_k) Z_k (Eq. 10) plus the box rows;
//   a4 clip    : the face plane a_F [x;1] = 0 (Eq. 12) starts as a square around the box
//                section.  Warp 0 cuts it by the 32 rows nearest to a point known to lie on
//                the face (the midpoint of the edge the cell was entered through, or the seed
//                point) in order of distance, each cut re-solving its two new vertices from
//                their planes (Eq. 11);
//   a5 check   : every thread then tests every row at every vertex of that polygon (Alg. 1
//                step 8 for the output); a violated row is cut in and the check repeated, so
//                the result is the clip by all rows whatever the candidates were;
//   a6 emit    : corners and edge planes to the face arena;
//   a7 march   : each edge on a neuron plane flips that neuron (Alg. 1 step 10) and pushes
//                the neighbour through the hash table (step 11).
//
// Two arithmetic modes.  kFP64: everything in FP64, a plane within delta of a vertex counts as
// satisfied (and as a degenerate event), as in the oracle.  kDF (mixed): the compose runs in
// double-float arithmetic on the FP32 pipes (TwoProd/TwoSum, the error-free transformations of
// Ogita, Rump & Oishi, "Accurate sum and dot product", 2005) and carries a rigorous bound on
// each row's error; polygon vertices are solved in FP64; every sign decision of the check is
// certified against the bounds (FP32 first, FP64 for the close calls) and a cell with an
// undecidable test is solved again in kFP64.
//
// Two schedules.  Persistent: a grid of resident blocks takes tickets (cell ids, in order)
// from a counter and waits, with a time limit, for the ticket's cell to be published; it stops
// when every handed-out cell is finished.  Levels: one launch per breadth-first level.
#include <algorithm>
#include <cuda_bf16.h>

#include "am_block.cuh"
#include "am_kernels.h"

namespace am {

// Threads per block and the minimum resident blocks per SM the compiler must allow for
// (register budget); both can be set at build time for launch-shape sweeps.
#ifndef AM_THREADS
#define AM_THREADS 256
#endif
#ifndef AM_MIN_BLOCKS
#define AM_MIN_BLOCKS 2
#endif
constexpr int kT = AM_THREADS;    // threads per block
constexpr int kNW = kT / 32;      // warps per block
constexpr int kMaxPoly = 64;      // polygon vertices in flight
constexpr int kNear = 32;         // rows clipped by warp 0 before the full check
constexpr int kPicks = kNear / kNW;   // candidates each warp contributes
static_assert(kT % 32 == 0 && kNW <= 32 && kNear % kNW == 0, "block shape");
constexpr int kMaxFix = 8;        // check / fix-up rounds
constexpr int kThreadPushWords = 8;   // keys up to this many 64-bit words are pushed by one thread per edge
constexpr float kU = 5.9604645e-8f;            // 2^-24
constexpr float kDfLoose = 1e-6f;              // certified row error (as a distance) beyond which kDF gives up
constexpr double kVertexTol = 1e-5;            // largest vertex error bound (relative) kept from kDF

enum { kFP64 = 0, kDF = 1 };

// Optional per-phase cycle counters (build with -DAM_PHASE_TIMERS): thread 0 of each block adds
// the clock64() cycles of each phase of each cell to counters[kPhase0 + phase * kCtrStride].
#ifdef AM_PHASE_TIMERS
#define AM_TICK(t) do { if (threadIdx.x == 0) (t) = clock64(); } while (0)
#define AM_PHASE(a, i, t0, t1) do { if (threadIdx.x == 0) atomicAdd((a).ar.counters + kPhase0 + (i) * kCtrStride, \
    (unsigned long long)((t1) - (t0))); } while (0)
#else
#define AM_TICK(t) do { } while (0)
#define AM_PHASE(a, i, t0, t1) do { } while (0)
#endif

// ------------------------------------------------------------------------------------------
// shared-memory layout

struct Lay {
    int mask, rows, err, rinv, carry, act, part, pv, pe, pf, vf, dvb, near, viol, sc, total;
};

__host__ __device__ inline int al16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline Lay march_layout(int max_n, int max_w)
{
    Lay s;
    const int nr = max_n + kBoxPlanes + kSquarePlanes;
    int o = 0;
    s.mask = o;  o = al16(o + ((max_n + 63) / 64) * 8);   // the whole key (kw 64-bit words)
    s.rows = o;  o = al16(o + nr * 32);                 // double[4] (FP64) or float[4] hi + float[4] lo (DF)
    s.err = o;   o = al16(o + nr * 4);
    s.rinv = o;  o = al16(o + nr * 4);
    s.carry = o; o = al16(o + max_w * 4);
    s.act = o;   o = al16(o + max_w * 4);
    s.part = o;  o = al16(o + kT * 40);
    s.pv = o;    o = al16(o + 2 * kMaxPoly * 3 * 8);
    s.pe = o;    o = al16(o + 2 * kMaxPoly * 4);
    s.pf = o;    o = al16(o + 2 * kMaxPoly * 3 * 4);
    s.vf = o;    o = al16(o + kMaxPoly * 4 * 4);
    s.dvb = o;   o = al16(o + kMaxPoly * 4);
    s.near = o;  o = al16(o + 2 * kNear * 4 + 2 * kNear * 4);
    s.viol = o;  o = al16(o + nr * 4);
    s.sc = o;    o = al16(o + 512);
    s.total = o;
    return s;
}

int march_smem_bytes(int max_n, int max_w) { return march_layout(max_n, max_w).total; }

// The proposal's scores use the compose scratch: 64 features + 2 hidden layers + 2 kT partials.
int proposal_max_hidden() { return (kT * 10 - 64 - 2 * kT) / 2; }

// The tensor-core compose keeps one layer's B fragments (16 bytes per lane per 16 input rows)
// in the low-part row array (16 bytes per row): 32 ceil(n_{l-1} / 16) <= max_n + 10 rows.
bool tc_fits(const int *width, int L, int max_n)
{
    for (int l = 2; l <= L; ++l)
        if (32 * ((width[l - 1] + 15) / 16) > max_n + kBoxPlanes + kSquarePlanes) return false;
    return true;
}

struct Sh {
    unsigned *mask;
    double *r64;            // FP64 rows [nr][4]
    float *rhi, *rlo;       // DF rows [nr][4] each
    float *err, *rinv, *carry;
    int *act;
    float *partf;
    double *partd;
    double (*pv)[kMaxPoly][3];
    int (*pe)[kMaxPoly];
    float (*pf)[kMaxPoly][3];   // kDF: the FP32 polygon of the candidate pass
    float (*vf)[4];             // final vertices in FP32 and max(1, |v|_inf)
    float *dvb;
    int *near_k, *near_w;
    float *near_d, *near_dw;
    int *viol;
    // scalars
    double *aF;             // 4 (FP64 value, or hi+lo of the DF value)
    float *aFhi, *aFlo;     // 4 + 4
    float *eF;              // 1
    int *si;                // 32 ints: 0 m, 1 buf, 2 status, 3 nviol, 4 amb, 5 ndeg, 6 emit, 7 ticket,
                            //          8 near count, 9 fix rounds, 10 a vertex too uncertain
    int *wsum;              // 32 ints
    unsigned long long *blk;   // per-block statistics, flushed once when the block exits:
                               // 0 solved, 1 empty, 2 degenerate, 3 fixups, 4 refined, 5 close calls,
                               // 6 cuts
};

__device__ inline Sh make_sh(unsigned char *base, int max_n, int max_w)
{
    const Lay L = march_layout(max_n, max_w);
    const int nr = max_n + kBoxPlanes + kSquarePlanes;
    Sh s;
    s.mask = (unsigned *)(base + L.mask);
    s.r64 = (double *)(base + L.rows);
    s.rhi = (float *)(base + L.rows);
    s.rlo = s.rhi + 4 * nr;
    s.err = (float *)(base + L.err);
    s.rinv = (float *)(base + L.rinv);
    s.carry = (float *)(base + L.carry);
    s.act = (int *)(base + L.act);
    s.partf = (float *)(base + L.part);
    s.partd = (double *)(base + L.part);
    s.pv = (double(*)[kMaxPoly][3])(base + L.pv);
    s.pe = (int(*)[kMaxPoly])(base + L.pe);
    s.pf = (float(*)[kMaxPoly][3])(base + L.pf);
    s.vf = (float(*)[4])(base + L.vf);
    s.dvb = (float *)(base + L.dvb);
    s.near_k = (int *)(base + L.near);
    s.near_d = (float *)(s.near_k + kNear);
    s.near_w = (int *)(s.near_d + kNear);
    s.near_dw = (float *)(s.near_w + kNear);
    s.viol = (int *)(base + L.viol);
    double *sc = (double *)(base + L.sc);
    s.aF = sc;                                   // 4 doubles
    s.aFhi = (float *)(sc + 4);                  // 4 floats
    s.aFlo = s.aFhi + 4;                         // 4 floats
    s.eF = s.aFlo + 4;                           // 1 float (+3 pad)
    s.si = (int *)(s.eF + 4);                    // 32 ints
    s.wsum = s.si + 32;                          // 32 ints
    s.blk = (unsigned long long *)(s.wsum + 32); // 8 x u64
    return s;
}

// ------------------------------------------------------------------------------------------
// arithmetic helpers

__device__ __forceinline__ bool bit_of(const unsigned *mask, int k) { return (mask[k >> 5] >> (k & 31)) & 1u; }

// s += a * z in double-float: (sh, sl) accumulates, a = ah + al, z = zh + zl.  The product
// ah*zh is split exactly (TwoProd with an FMA), the sum with TwoSum; the small cross terms and
// every error term go to sl.  Explicit _rn intrinsics keep the compiler from fusing them.
__device__ __forceinline__ void df_fma(float &sh, float &sl, float ah, float al, float zh, float zl)
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

// (sh, sl) += (bh, bl) (TwoSum on the high parts)
__device__ __forceinline__ void df_add(float &sh, float &sl, float bh, float bl)
{
    const float t = __fadd_rn(sh, bh);
    const float bp = __fsub_rn(t, sh);
    const float te = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(bh, bp));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(te, bl));
}

// renormalise so that |lo| <= ulp(hi) / 2 (Fast2Sum)
__device__ __forceinline__ void df_norm(float &h, float &l)
{
    const float s = __fadd_rn(h, l);
    l = __fsub_rn(l, __fsub_rn(s, h));
    h = s;
}

// gamma-style coefficient of the double-float dot product bound: 2 (m + 4)^2 u^2
__device__ __forceinline__ float df_gamma(int m) { return 2.0f * (float)(m + 4) * (float)(m + 4) * kU * kU; }

// row k as FP64 (both modes; in kDF hi + lo is exact in FP64)
template <int M>
__device__ __forceinline__ void row64(const Sh &s, int k, double *r)
{
    if (M == kFP64) {
        r[0] = s.r64[4 * k]; r[1] = s.r64[4 * k + 1]; r[2] = s.r64[4 * k + 2]; r[3] = s.r64[4 * k + 3];
    } else {
        for (int c = 0; c < 4; ++c) r[c] = (double)s.rhi[4 * k + c] + (double)s.rlo[4 * k + c];
    }
}

// ------------------------------------------------------------------------------------------
// a2 on the tensor cores: hidden layers 2..L of the compose as split-BF16 products

// D (16 x 8, FP32) += A (16 x 16, BF16, row) * B (16 x 8, BF16, col); fragments as in the PTX
// ISA's mma.m16n8k16 layouts (a: 4 x b32, b: 2 x b32, lower element in the lower half)
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint4 &a, const uint2 &b)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ unsigned bf16_bits(float x)
{
    return (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}

constexpr int kTcTiles = 4;         // 16-row output tiles a warp accumulates at once

// Z_l = W_l diag(s_{l-1}) Z_{l-1} + C_l for l = 2..L on the tensor cores.  Z_{l-1} (FP32 rows,
// sign-adjusted, in s.rhi; inactive rows zero) is split into three BF16 parts and laid out as
// B1 = [Z_hi | Z_mid] and B2 = [Z_lo | 0] (16 x 8 fragments); W_l comes as three BF16 parts.
// Four MMAs per tile: (W_hi + W_mid + W_lo) B1 + W_hi B2, whose two column halves sum to
// W (Z_hi + Z_mid) + W_hi Z_lo: the dropped products and split residuals are below 2^-26 |W||Z|,
// so the FP32 accumulation dominates.  The B fragments live in s.rlo, unused by this path
// (it is zeroed before return: tensor-core rows have no low part).
// Error estimate per row m (l1 over its 4 coefficients), not a bound:
//   8 (2.8 2^-24 sqrt(T) + 2^-25) max_j |W_mj| sum_c |z_c|_2  +  |W_m|_2 rms(e_{l-1}),  T = 4 Kt
// (random-sign model of the accumulation over T MMAs, each product's share bounded through
// max|W_mj| and the column norm; the previous rows' estimates propagate by root mean square,
// without a new factor, so the safety does not compound with depth).
__device__ __noinline__ void compose_tc_layers(const NetDev &net, const Sh &s, int nr)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, g = lane >> 2, t4 = lane & 3;
    uint4 *Bf = reinterpret_cast<uint4 *>(s.rlo);   // per (kt, lane): B1 (x, y), B2 (z, w)
    float *red = reinterpret_cast<float *>(s.wsum);   // 0..3: sum z_c^2, 4: sum e^2 (no scans here)
    for (int l = 2; l <= net.L; ++l) {
        const int np = net.width[l - 1], nl = net.width[l], rp = net.row0[l - 1], rl = net.row0[l];
        const int Kt = (np + 15) >> 4, Mt = (nl + 15) >> 4;
        if (tid < 8) red[tid] = 0.0f;
        __syncthreads();
        // B fragments: item (kt, lane') holds rows kt*16 + 2t' + {0, 1, 8, 9} of column g'
        for (int it = tid; it < Kt * 32; it += kT) {
            const int kt = it >> 5, gg = (it & 31) >> 2, tt = it & 3;
            const int c = gg & 3;
            const bool second = gg >= 4;              // columns 4..7: Z_mid in B1, zero in B2
            unsigned v1[4], v2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = kt * 16 + 2 * tt + (q & 1) + (q >> 1) * 8;
                float z = 0.0f;
                if (k < np && bit_of(s.mask, rp + k)) z = -s.rhi[4 * (rp + k) + c];   // active: z = -row
                const float zh = __bfloat162float(__float2bfloat16_rn(z));
                const float zm = __bfloat162float(__float2bfloat16_rn(z - zh));
                v1[q] = bf16_bits(second ? zm : zh);
                v2[q] = second ? 0u : bf16_bits((z - zh) - zm);
            }
            Bf[it] = make_uint4(v1[0] | (v1[1] << 16), v1[2] | (v1[3] << 16), v2[0] | (v2[1] << 16),
                                v2[2] | (v2[3] << 16));
        }
        {
            float z2[4] = {0.0f, 0.0f, 0.0f, 0.0f}, e2 = 0.0f;
            for (int k = tid; k < np; k += kT)
                if (bit_of(s.mask, rp + k)) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) z2[c] = fmaf(s.rhi[4 * (rp + k) + c], s.rhi[4 * (rp + k) + c], z2[c]);
                    e2 = fmaf(s.err[rp + k], s.err[rp + k], e2);
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int c = 0; c < 4; ++c) z2[c] += __shfl_xor_sync(0xffffffffu, z2[c], o);
                e2 += __shfl_xor_sync(0xffffffffu, e2, o);
            }
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < 4; ++c) atomicAdd(red + c, z2[c]);
                atomicAdd(red + 4, e2);
            }
        }
        __syncthreads();
        const float zn = sqrtf(red[0]) + sqrtf(red[1]) + sqrtf(red[2]) + sqrtf(red[3]);
        const float erms = sqrtf(red[4] / (float)np);
        const float kloc = 8.0f * (2.8f * 5.9604644775390625e-8f * sqrtf((float)(4 * Kt)) + 2.98023223876953125e-8f);
        const uint4 *Wf = net.Wf[l];
        const float *wn = net.wn[l];
        for (int mt0 = wid; mt0 < Mt; mt0 += kNW * kTcTiles) {
            float acc[kTcTiles][4];
#pragma unroll
            for (int i = 0; i < kTcTiles; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0f;
            for (int kt = 0; kt < Kt; ++kt) {
                const uint4 bb = Bf[kt * 32 + lane];
                const uint2 b1 = make_uint2(bb.x, bb.y), b2 = make_uint2(bb.z, bb.w);
#pragma unroll
                for (int i = 0; i < kTcTiles; ++i) {
                    const int mt = mt0 + i * kNW;
                    if (mt < Mt) {
                        const uint4 *tp = Wf + ((size_t)mt * Kt + kt) * 96;
                        const uint4 ah = __ldg(tp + lane), am = __ldg(tp + 32 + lane), al = __ldg(tp + 64 + lane);
                        mma_bf16_16816(acc[i], ah, b1);
                        mma_bf16_16816(acc[i], am, b1);
                        mma_bf16_16816(acc[i], al, b1);
                        mma_bf16_16816(acc[i], ah, b2);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < kTcTiles; ++i) {
                const int mt = mt0 + i * kNW;
                if (mt >= Mt) continue;                  // warp-uniform
                float o[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) o[q] = acc[i][q] + __shfl_xor_sync(0xffffffffu, acc[i][q], 2);
                if (t4 < 2) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {        // rows g and g + 8
                        const int m = mt * 16 + g + 8 * h;
                        if (m >= nl) continue;
                        const int r = rl + m;
                        const float sg = bit_of(s.mask, r) ? -1.0f : 1.0f;
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const int c = 2 * t4 + j;
                            const float v = o[2 * h + j] + (net.Clhi[l][4 * m + c] + net.Cllo[l][4 * m + c]);
                            s.rhi[4 * r + c] = sg * v;
                        }
                        if (t4 == 0) s.err[r] = fmaf(kloc * wn[2 * m + 1], zn, wn[2 * m] * erms);
                    }
                }
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < 4 * nr; i += kT) s.rlo[i] = 0.0f;
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// a2/a3: compose the rows of every neuron of the cell, and a_F

// The residual shortcut of layer l (Sec. 5.1) for its row k, FP64: a += sum_j S_kj H_src[j] with
// H_src = diag(g) Z_src (g = 1 on active units, the slope on the others) and the stored row
// (1 - 2 s) Z, so H_src[j] = -row_j when unit j is active and slope * row_j otherwise; S = null
// is the identity (H_src[k]).
__device__ __forceinline__ void add_shortcut(const NetDev &net, const Sh &s, int l, int k, double &a0, double &a1,
                                             double &a2, double &a3)
{
    const int src = net.sc_src[l];
    if (src <= 0) return;
    const int rs = net.row0[src], ns = net.width[src];
    const double *S = net.sc_S[l];
    const int j0 = S ? 0 : k, j1 = S ? ns : k + 1;
    for (int j = j0; j < j1; ++j) {
        const double w = S ? __ldg(S + (size_t)k * ns + j) : 1.0;
        const int r = rs + j;
        const double f = w * (bit_of(s.mask, r) ? -1.0 : net.slope);
        if (f == 0.0) continue;
        const double *z = s.r64 + 4 * r;
        a0 += f * z[0]; a1 += f * z[1]; a2 += f * z[2]; a3 += f * z[3];
    }
}

template <int M>
__device__ __forceinline__ void compose(const NetDev &net, const Sh &s, bool tc, int nrows)
{
    const int tid = threadIdx.x;
    // layer 1: Z_1 = C_1 (cell independent)
    {
        const int n1 = net.width[1];
        for (int k = tid; k < n1; k += kT) {
            const bool act = bit_of(s.mask, k);
            if (M == kFP64) {
                const double sg = act ? -1.0 : 1.0;
                for (int c = 0; c < 4; ++c) s.r64[4 * k + c] = sg * net.Cl[1][4 * k + c];
            } else {
                const float sg = act ? -1.0f : 1.0f;
                float l1 = 0.0f;
                for (int c = 0; c < 4; ++c) {
                    const float h = net.Clhi[1][4 * k + c], l = net.Cllo[1][4 * k + c];
                    s.rhi[4 * k + c] = sg * h;
                    s.rlo[4 * k + c] = sg * l;
                    l1 += fabsf(h);
                }
                // representation of C: double-float, or FP32 alone on the tensor-core path
                s.err[k] = tc ? kU * l1 * 1.01f : 2.0f * kU * kU * l1 * 1.01f;
            }
        }
    }
    __syncthreads();
    if (M == kDF && tc) compose_tc_layers(net, s, nrows);
    for (int l = (M == kDF && tc) ? net.L + 1 : 2; l <= net.L; ++l) {
        const int np = net.width[l - 1], nl = net.width[l], rp = net.row0[l - 1], rl = net.row0[l];
        const int S = nl >= kT ? 1 : kT / nl;
        // active list of layer l-1 (diag(s_{l-1}) selects these rows); with a leaky ReLU every
        // row takes part, the inactive ones scaled by the slope (diag(s + slope (1 - s)))
        const bool leaky = M == kFP64 && net.slope != 0.0;
        int nact = 0;
        for (int base = 0; base < np; base += kT) {
            const int j = base + tid;
            const int f = (j < np) ? (leaky ? 1 : (int)bit_of(s.mask, rp + j)) : 0;
            int tot;
            const int pos = block_scan_excl(f, s.wsum, &tot);
            if (f) s.act[nact + pos] = j;
            nact += tot;
        }
        __syncthreads();                     // the active list is read by every thread below
        float g = 0.0f;
        if (M == kDF) {
            g = df_gamma(nact + S + 2);
            // carry_t = e_j + g |z_j|_1 for the t-th active row j of layer l-1
            for (int t = tid; t < nact; t += kT) {
                const int r = rp + s.act[t];
                const float l1 = fabsf(s.rhi[4 * r]) + fabsf(s.rhi[4 * r + 1]) + fabsf(s.rhi[4 * r + 2]) +
                                 fabsf(s.rhi[4 * r + 3]);
                s.carry[t] = __fmaf_ru(g, l1 * 1.001f, s.err[r]);
            }
        }
        __syncthreads();
        for (int item = tid; item < nl * S; item += kT) {
            const int k = item % nl, sp = item / nl;
            if (M == kFP64) {
                const double *AT = net.AT[l];
                double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                if (leaky) {
                    // active: z = -row (weight 1); inactive: z = +row, weight slope
                    const double sl = net.slope;
                    for (int t = sp; t < nact; t += S) {
                        const int j = s.act[t];
                        double w = __ldg(AT + (size_t)j * nl + k);
                        if (!bit_of(s.mask, rp + j)) w *= -sl;
                        const double *z = s.r64 + 4 * (rp + j);
                        a0 -= w * z[0]; a1 -= w * z[1]; a2 -= w * z[2]; a3 -= w * z[3];
                    }
                } else {
#pragma unroll 4
                    for (int t = sp; t < nact; t += S) {
                        const int j = s.act[t];
                        const double w = __ldg(AT + (size_t)j * nl + k);
                        const double *z = s.r64 + 4 * (rp + j);          // active: z = -row
                        a0 -= w * z[0]; a1 -= w * z[1]; a2 -= w * z[2]; a3 -= w * z[3];
                    }
                }
                if (S == 1) {
                    add_shortcut(net, s, l, k, a0, a1, a2, a3);
                    const double sg = bit_of(s.mask, rl + k) ? -1.0 : 1.0;
                    const double *C = net.Cl[l] + 4 * k;
                    double *r = s.r64 + 4 * (rl + k);
                    r[0] = sg * (a0 + C[0]); r[1] = sg * (a1 + C[1]); r[2] = sg * (a2 + C[2]); r[3] = sg * (a3 + C[3]);
                } else {
                    double *p = s.partd + 4 * item;
                    p[0] = a0; p[1] = a1; p[2] = a2; p[3] = a3;
                }
            } else {
                const float *Ah = net.AThi[l], *Al = net.ATlo[l];
                float h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f, l0 = 0.f, l1 = 0.f, l2 = 0.f, l3 = 0.f, eb = 0.f;
#pragma unroll 4
                for (int t = sp; t < nact; t += S) {
                    const int j = s.act[t];
                    const float ah = __ldg(Ah + (size_t)j * nl + k), al = __ldg(Al + (size_t)j * nl + k);
                    const float4 zh = *reinterpret_cast<const float4 *>(s.rhi + 4 * (rp + j));   // z = -row
                    const float4 zl = *reinterpret_cast<const float4 *>(s.rlo + 4 * (rp + j));
                    df_fma(h0, l0, ah, al, -zh.x, -zl.x);
                    df_fma(h1, l1, ah, al, -zh.y, -zl.y);
                    df_fma(h2, l2, ah, al, -zh.z, -zl.z);
                    df_fma(h3, l3, ah, al, -zh.w, -zl.w);
                    eb = __fmaf_ru(fabsf(ah), s.carry[t], eb);
                }
                if (S == 1) {
                    const float *Ch = net.Clhi[l] + 4 * k, *Cc = net.Cllo[l] + 4 * k;
                    df_add(h0, l0, Ch[0], Cc[0]); df_add(h1, l1, Ch[1], Cc[1]);
                    df_add(h2, l2, Ch[2], Cc[2]); df_add(h3, l3, Ch[3], Cc[3]);
                    df_norm(h0, l0); df_norm(h1, l1); df_norm(h2, l2); df_norm(h3, l3);
                    const float sg = bit_of(s.mask, rl + k) ? -1.0f : 1.0f;
                    *reinterpret_cast<float4 *>(s.rhi + 4 * (rl + k)) = make_float4(sg * h0, sg * h1, sg * h2, sg * h3);
                    *reinterpret_cast<float4 *>(s.rlo + 4 * (rl + k)) = make_float4(sg * l0, sg * l1, sg * l2, sg * l3);
                    const float cl1 = fabsf(Ch[0]) + fabsf(Ch[1]) + fabsf(Ch[2]) + fabsf(Ch[3]);
                    s.err[rl + k] = __fmaf_ru(g, cl1, eb) * 1.01f;
                } else {
                    float *p = s.partf + 9 * item;
                    p[0] = h0; p[1] = h1; p[2] = h2; p[3] = h3; p[4] = l0; p[5] = l1; p[6] = l2; p[7] = l3; p[8] = eb;
                }
            }
        }
        __syncthreads();
        if (S > 1) {
            for (int k = tid; k < nl; k += kT) {
                if (M == kFP64) {
                    const double *C = net.Cl[l] + 4 * k;
                    double a0 = C[0], a1 = C[1], a2 = C[2], a3 = C[3];
                    for (int sp = 0; sp < S; ++sp) {
                        const double *p = s.partd + 4 * (sp * nl + k);
                        a0 += p[0]; a1 += p[1]; a2 += p[2]; a3 += p[3];
                    }
                    add_shortcut(net, s, l, k, a0, a1, a2, a3);
                    const double sg = bit_of(s.mask, rl + k) ? -1.0 : 1.0;
                    double *r = s.r64 + 4 * (rl + k);
                    r[0] = sg * a0; r[1] = sg * a1; r[2] = sg * a2; r[3] = sg * a3;
                } else {
                    const float *Ch = net.Clhi[l] + 4 * k, *Cc = net.Cllo[l] + 4 * k;
                    float h0 = Ch[0], h1 = Ch[1], h2 = Ch[2], h3 = Ch[3];
                    float l0 = Cc[0], l1 = Cc[1], l2 = Cc[2], l3 = Cc[3];
                    float eb = 0.0f;
                    for (int sp = 0; sp < S; ++sp) {
                        const float *p = s.partf + 9 * (sp * nl + k);
                        df_add(h0, l0, p[0], p[4]); df_add(h1, l1, p[1], p[5]);
                        df_add(h2, l2, p[2], p[6]); df_add(h3, l3, p[3], p[7]);
                        eb = __fadd_ru(eb, p[8]);
                    }
                    df_norm(h0, l0); df_norm(h1, l1); df_norm(h2, l2); df_norm(h3, l3);
                    const float sg = bit_of(s.mask, rl + k) ? -1.0f : 1.0f;
                    *reinterpret_cast<float4 *>(s.rhi + 4 * (rl + k)) = make_float4(sg * h0, sg * h1, sg * h2, sg * h3);
                    *reinterpret_cast<float4 *>(s.rlo + 4 * (rl + k)) = make_float4(sg * l0, sg * l1, sg * l2, sg * l3);
                    const float cl1 = fabsf(Ch[0]) + fabsf(Ch[1]) + fabsf(Ch[2]) + fabsf(Ch[3]);
                    s.err[rl + k] = __fmaf_ru(g, cl1, eb) * 1.01f;
                }
            }
            __syncthreads();
        }
    }
    // a_F = w_out^T diag(s_L) Z_L + [0 | b_out]  (Cor. 1, Eq. 8)
    if (M == kFP64 && net.M >= 2) {
        // final max pooling (Sec. 5.2): a_F(i) of every head into row n_units + i, then the face
        // plane a_F(j) of the cell's pooled index j and the pooling rows a_F(i) - a_F(j)
        const int nL = net.width[net.L], rL = net.row0[net.L];
        for (int i = 0; i < net.M; ++i) {
            const double *wh = net.w_heads + (size_t)i * nL;
            double f[4] = {0.0, 0.0, 0.0, 0.0};
            for (int k = tid; k < nL; k += kT) {
                const double w = bit_of(s.mask, rL + k) ? wh[k] : -net.slope * wh[k];
                if (w != 0.0)
                    for (int c = 0; c < 4; ++c) f[c] -= w * s.r64[4 * (rL + k) + c];
            }
            for (int c = 0; c < 4; ++c) f[c] = warp_sum(f[c]);
            if ((tid & 31) == 0)
                for (int c = 0; c < 4; ++c) s.partd[4 * (tid >> 5) + c] = f[c];
            __syncthreads();
            if (tid == 0) {
                double F[4] = {0.0, 0.0, 0.0, net.b_heads[i]};
                for (int w = 0; w < kNW; ++w)
                    for (int c = 0; c < 4; ++c) F[c] += s.partd[4 * w + c];
                for (int c = 0; c < 4; ++c) s.r64[4 * (net.n_units + i) + c] = F[c];
            }
            __syncthreads();
        }
        if (tid == 0) {
            int j = 0;
            for (int i = 0; i < net.M; ++i)
                if (bit_of(s.mask, net.n_units + i)) { j = i; break; }
            for (int c = 0; c < 4; ++c) s.aF[c] = s.r64[4 * (net.n_units + j) + c];
            s.eF[0] = 0.0f;
        }
        __syncthreads();
        if (tid < net.M)
            for (int c = 0; c < 4; ++c) s.r64[4 * (net.n_units + tid) + c] -= s.aF[c];
        __syncthreads();
        return;
    }
    {
        const int nL = net.width[net.L], rL = net.row0[net.L];
        if (M == kFP64) {
            double f[4] = {0.0, 0.0, 0.0, 0.0};
            for (int k = tid; k < nL; k += kT) {
                // active: row = -Z (weight 1); inactive: row = +Z, weight slope (0 for a ReLU)
                const double w = bit_of(s.mask, rL + k) ? net.w_out[k] : -net.slope * net.w_out[k];
                if (w != 0.0)
                    for (int c = 0; c < 4; ++c) f[c] -= w * s.r64[4 * (rL + k) + c];
            }
            for (int c = 0; c < 4; ++c) f[c] = warp_sum(f[c]);
            if ((tid & 31) == 0)
                for (int c = 0; c < 4; ++c) s.partd[4 * (tid >> 5) + c] = f[c];
            __syncthreads();
            if (tid == 0) {
                double F[4] = {0.0, 0.0, 0.0, net.b_out};
                for (int w = 0; w < kNW; ++w)
                    for (int c = 0; c < 4; ++c) F[c] += s.partd[4 * w + c];
                for (int c = 0; c < 4; ++c) s.aF[c] = F[c];
                s.eF[0] = 0.0f;
            }
        } else {
            // one warp, lanes over the last layer, double-float with a bound
            if (tid < 32) {
                int cnt = 0;
                for (int k = tid; k < nL; k += 32) cnt += bit_of(s.mask, rL + k);
                for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
                const float g = df_gamma(cnt + 40);
                float h[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f}, eb = 0.0f, e2 = 0.0f;
                for (int k = tid; k < nL; k += 32) {
                    if (!bit_of(s.mask, rL + k)) continue;
                    const float wh = net.w_out_hi[k], wl = net.w_out_lo[k];
                    const float *zh = s.rhi + 4 * (rL + k), *zl = s.rlo + 4 * (rL + k);
                    float l1 = 0.0f;
                    for (int c = 0; c < 4; ++c) {
                        df_fma(h[c], lo[c], wh, wl, -zh[c], -zl[c]);
                        l1 += fabsf(zh[c]);
                    }
                    if (tc) {           // this product's rounding (bound) + propagated estimates (rss)
                        eb = __fmaf_ru(fabsf(wh), g * l1 * 1.001f, eb);
                        e2 = fmaf(wh * s.err[rL + k], wh * s.err[rL + k], e2);
                    } else {
                        eb = __fmaf_ru(fabsf(wh), __fmaf_ru(g, l1 * 1.001f, s.err[rL + k]), eb);
                    }
                }
#pragma unroll 1
                for (int o = 16; o > 0; o >>= 1) {
                    for (int c = 0; c < 4; ++c) {
                        const float oh = __shfl_xor_sync(0xffffffffu, h[c], o);
                        const float ol = __shfl_xor_sync(0xffffffffu, lo[c], o);
                        df_add(h[c], lo[c], oh, ol);
                    }
                    eb = __fadd_ru(eb, __shfl_xor_sync(0xffffffffu, eb, o));
                    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
                }
                if (tc) eb += 2.0f * sqrtf(e2);
                if (tid == 0) {
                    const float bh = (float)net.b_out, bl = (float)(net.b_out - (double)bh);
                    df_add(h[3], lo[3], bh, bl);
                    float l1 = fabsf(bh);
                    for (int c = 0; c < 4; ++c) {
                        df_norm(h[c], lo[c]);
                        s.aFhi[c] = h[c];
                        s.aFlo[c] = lo[c];
                        s.aF[c] = (double)h[c] + (double)lo[c];
                    }
                    s.eF[0] = __fmaf_ru(g, l1, eb) * 1.01f;
                }
            }
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// polygon helpers (warp 0)

template <class R>
__device__ __forceinline__ R pdist(const R *r, R ri, const R *v)
{
    return (r[0] * v[0] + r[1] * v[1] + r[2] * v[2] + r[3]) * ri;
}

// One cut of the polygon P[buf] (edge planes E[buf], m vertices) by row k, warp-parallel.  A
// vertex is cut off when its distance from row k's plane exceeds tol.  The two new vertices are
// re-solved from their planes and the face plane aF.  Returns the new vertex count (0 = empty,
// -1 = inconsistent or overflow); *swapped tells whether the result went to buffer buf ^ 1.
// row q in the vertex type R: FP64 rows (any mode) or the FP32 high parts (kDF heuristic pass)
template <class R, int M>
__device__ __forceinline__ void fetch_row(const Sh &s, int q, R *r)
{
    if constexpr (sizeof(R) == 8) {
        row64<M>(s, q, (double *)r);
    } else {
        r[0] = s.rhi[4 * q]; r[1] = s.rhi[4 * q + 1]; r[2] = s.rhi[4 * q + 2]; r[3] = s.rhi[4 * q + 3];
    }
}

template <class R, int M>
__device__ __forceinline__ int warp_cut(const Sh &s, R (*P)[kMaxPoly][3], int m, int buf, int k, R tol, const R *aF,
                                        bool *swapped)
{
    int (*E)[kMaxPoly] = s.pe;
    const int lane = threadIdx.x & 31;
    *swapped = false;
    R rk[4];
    fetch_row<R, M>(s, k, rk);
    const R rn = sqrt(rk[0] * rk[0] + rk[1] * rk[1] + rk[2] * rk[2]);
    if (rn == R(0)) return m;
    const R ri = R(1) / rn;
    const bool o0 = lane < m && pdist(rk, ri, P[buf][lane]) > tol;
    const bool o1 = lane + 32 < m && pdist(rk, ri, P[buf][lane + 32]) > tol;
    const unsigned long long out = (unsigned long long)__ballot_sync(0xffffffffu, o0) |
                                   ((unsigned long long)__ballot_sync(0xffffffffu, o1) << 32);
    const int nout = __popcll(out);
    if (nout == 0) return m;
    if (nout == m) return 0;
    int ia = -1, ib = -1;
    for (int i = lane; i < m; i += 32) {
        const bool oi = (out >> i) & 1ull;
        if (oi && !((out >> ((i + m - 1) % m)) & 1ull)) ia = i;
        if (oi && !((out >> ((i + 1) % m)) & 1ull)) ib = i;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ia = max(ia, __shfl_xor_sync(0xffffffffu, ia, o));
        ib = max(ib, __shfl_xor_sync(0xffffffffu, ib, o));
    }
    if (ia < 0 || ib < 0 || ((ib - ia + m) % m) + 1 != nout) return -1;
    const int nin = m - nout;
    if (nin + 2 > kMaxPoly) return -1;
    const int nb = buf ^ 1;
    const int ea = E[buf][(ia + m - 1) % m], eb = E[buf][ib];
    for (int i = lane; i < m; i += 32) {                 // the kept run b+1 .. a-1, in order
        if ((out >> i) & 1ull) continue;
        const int ni = (i - (ib + 1) + m) % m;
        P[nb][ni][0] = P[buf][i][0]; P[nb][ni][1] = P[buf][i][1]; P[nb][ni][2] = P[buf][i][2];
        E[nb][ni] = E[buf][i];
    }
    bool ok = true;
    if (lane < 2) {
        R pa[4], pb[4], v[3];
        fetch_row<R, M>(s, lane == 0 ? ea : k, pa);
        fetch_row<R, M>(s, lane == 0 ? k : eb, pb);
        ok = solve3<R>(pa, pb, aF, v, nullptr);
        P[nb][nin + lane][0] = v[0]; P[nb][nin + lane][1] = v[1]; P[nb][nin + lane][2] = v[2];
        E[nb][nin + lane] = lane == 0 ? k : eb;
    }
    ok = __all_sync(0xffffffffu, ok);
    __syncwarp();
    *swapped = true;
    return ok ? nin + 2 : -1;
}

// kDF: the final vertices in FP64 from the double-float rows, with the bound dv on how far the
// exact vertex (exact rows) can be, |v* - v|_inf <= |M^-1|_inf max(e_a, e_b, e_F) max(1,|v|) (1.1).
__device__ __forceinline__ void df_final_vertices(const Sh &s, int m, int buf, double vtol)
{
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < m; i += 32) {
        const int ea = s.pe[buf][(i + m - 1) % m], eb = s.pe[buf][i];
        double ra[4], rb[4], v[3], inorm = 0.0;
        row64<kDF>(s, ea, ra);
        row64<kDF>(s, eb, rb);
        const bool ok = solve3<double>(ra, rb, s.aF, v, &inorm);
        const double X = fmax(1.0, fmax(fabs(v[0]), fmax(fabs(v[1]), fabs(v[2]))));
        const double e = fmax((double)s.err[ea], fmax((double)s.err[eb], (double)s.eF[0]));
        s.pv[buf][i][0] = v[0]; s.pv[buf][i][1] = v[1]; s.pv[buf][i][2] = v[2];
        s.dvb[i] = ok ? (float)(inorm * e * X * 1.1 + 4e-16 * X) * 1.01f : 3.0e38f;
        if (s.dvb[i] > vtol * X) s.si[10] = 1;           // this vertex is not known well enough
    }
    __syncwarp();
}

// ------------------------------------------------------------------------------------------
// learned proposal: scores of every neuron row for this cell (block-wide forward pass)

// Features: entry point (3), unit face-plane normal (3), plane offset (1), active fraction of
// each hidden layer (L).  Scores go to z[0..N) (logits; larger = more likely an edge plane).
// y = W x for one cell, W^T stored as n_in rows of n_pairs BF16 pairs (row stride 2 n_pairs).
// Threads take output pairs; when there are fewer pairs than threads the j range is split G
// ways and the partial sums go to part (G x 2 n_pairs floats).  G == 1: y = act(W x + b).
__device__ __forceinline__ void gemv_bf16x2(const __nv_bfloat16 *wt, int n_pairs, int n_in, int n_out,
                                            const float *x, const float *b, bool relu, float *y, float *part, int G)
{
    const __nv_bfloat162 *w = reinterpret_cast<const __nv_bfloat162 *>(wt);
    for (int q = threadIdx.x; q < n_pairs * G; q += kT) {
        const int pr = q % n_pairs, g = q / n_pairs;
        const int j0 = g * n_in / G, j1 = (g + 1) * n_in / G;
        float a0 = 0.0f, a1 = 0.0f;
        const __nv_bfloat162 *wp = w + pr;
#pragma unroll 32
        for (int j = j0; j < j1; ++j) {         // 32 weight loads in flight: the weights stream from L2
            const float2 wf = __bfloat1622float2(wp[(size_t)j * n_pairs]);
            const float xj = x[j];
            a0 = fmaf(wf.x, xj, a0);
            a1 = fmaf(wf.y, xj, a1);
        }
        const int o = 2 * pr;
        if (G == 1) {
            a0 += b[o];
            y[o] = relu ? fmaxf(a0, 0.0f) : a0;
            if (o + 1 < n_out) {
                a1 += b[o + 1];
                y[o + 1] = relu ? fmaxf(a1, 0.0f) : a1;
            }
        } else {
            part[g * 2 * n_pairs + o] = a0;
            part[g * 2 * n_pairs + o + 1] = a1;
        }
    }
    if (G > 1) {
        __syncthreads();
        for (int o = threadIdx.x; o < n_out; o += kT) {
            float a = b[o];
            for (int g = 0; g < G; ++g) a += part[g * 2 * n_pairs + o];
            y[o] = relu ? fmaxf(a, 0.0f) : a;
        }
    }
}

// Learned proposal (no counterpart in the paper): sigmoid-free scores z[0:N] of every neuron for
// this cell, from its entry point, the unit normal and offset of a_F and the per-layer active
// fractions of its pattern.  Hidden widths are even (BF16 pairs); W3^T rows are padded to even.
__device__ void proposal_scores(const MarchArgs &a, const NetDev &net, int64_t cell, const Sh &s, float *z)
{
    const ProposalView &P = a.prop;
    const int tid = threadIdx.x, H = P.hidden, O = P.n_out, I = P.n_in;
    float *x = s.partf;            // the compose partial sums are free here
    float *h1 = x + 64, *h2 = h1 + H, *part = h2 + H;
    if (tid == 0) {
        x[0] = __ldcg(a.ar.entry_pt + cell * 3);
        x[1] = __ldcg(a.ar.entry_pt + cell * 3 + 1);
        x[2] = __ldcg(a.ar.entry_pt + cell * 3 + 2);
        const double *F = s.aF;
        const double inv = 1.0 / sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
        x[3] = (float)(F[0] * inv); x[4] = (float)(F[1] * inv); x[5] = (float)(F[2] * inv); x[6] = (float)(F[3] * inv);
        for (int l = 1; l <= net.L; ++l) {
            const int r0 = net.row0[l], n = net.width[l];
            int cnt = 0;
            for (int w = r0 >> 5; w <= (r0 + n - 1) >> 5; ++w) {
                unsigned bits = s.mask[w];
                const int lo = max(r0 - 32 * w, 0), hi = min(r0 + n - 32 * w, 32);
                bits &= (hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
                cnt += __popc(bits);
            }
            x[6 + l] = (float)cnt / (float)n;
        }
    }
    __syncthreads();
    for (int t = tid; t < H; t += kT) {
        float acc = P.b1[t];
        for (int i = 0; i < I; ++i) acc = fmaf(__bfloat162float(P.w1[(size_t)t * I + i]), x[i], acc);
        h1[t] = fmaxf(acc, 0.0f);
    }
    __syncthreads();
    const int H2 = H >> 1, O2 = (O + 1) >> 1;
    gemv_bf16x2(P.w2t, H2, H, H, h1, P.b2, true, h2, part, H2 >= kT ? 1 : kT / H2);
    __syncthreads();
    gemv_bf16x2(P.w3t, O2, H, O, h2, P.b3, false, z, part, O2 >= kT ? 1 : kT / O2);
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// one cell

struct CellOut {
    int emit;        // corners written (0 = empty)
    int ambiguous;   // kDF: an undecidable sign test; nothing written
};

template <int M>
__device__ __noinline__ CellOut solve_cell(const MarchArgs &a, const NetDev &net, int64_t cell, const Sh &s)
{
    const Arena &ar = a.ar;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int N = net.N, NC = N + kBoxPlanes;          // checked rows: neurons + box
    long long tp0 = 0, tp1 = 0, tp2 = 0, tp2a = 0, tp3a = 0, tp3 = 0, tp4 = 0, tp4a = 0, tp5 = 0;
    AM_TICK(tp0);
    if (a.rows_in) {
        // rows composed beforehand on the tensor cores, as FP32 pairs (the hi words [hi x 4] of
        // rows 0..N, then their lo words [lo x 4])
        // (signs as compose<M>, a_F last).  The pairs are the rows: the double-float tests are
        // certified against them with no further row error, as FP64 tests take FP64 rows.
        const float4 *src = reinterpret_cast<const float4 *>(a.rows_in) + (cell - a.begin) * (int64_t)(N + 1) * 2;
        for (int k = tid; k < N; k += kT) {
            const float4 h = __ldcs(src + k), l = __ldcs(src + (N + 1) + k);
            if (M == kFP64) {
                double *r = s.r64 + 4 * k;
                r[0] = (double)h.x + (double)l.x; r[1] = (double)h.y + (double)l.y;
                r[2] = (double)h.z + (double)l.z; r[3] = (double)h.w + (double)l.w;
            } else {
                *reinterpret_cast<float4 *>(s.rhi + 4 * k) = h;
                *reinterpret_cast<float4 *>(s.rlo + 4 * k) = l;
                s.err[k] = 0.0f;
            }
        }
        if (tid < 4) {
            const float h = reinterpret_cast<const float *>(src + N)[tid];
            const float l = reinterpret_cast<const float *>(src + 2 * N + 1)[tid];
            s.aF[tid] = (double)h + (double)l;
            if (M == kDF) { s.aFhi[tid] = h; s.aFlo[tid] = l; }
        }
        if (tid == 0) s.eF[0] = 0.0f;
        __syncthreads();
    } else {
        compose<M>(net, s, false, a.max_n + kBoxPlanes + kSquarePlanes);
    }
    AM_TICK(tp1);

    // box rows (exact), frame and the initial square (thread 0)
    // (kDF: the pairs are stored as they are, exact FP32 words: the normal's components are
    // 0 and +-1 and the offset is the host's split of the box, so no conversion runs here)
    for (int i = tid; i < kBoxPlanes; i += kT) {
        const int ax = i >> 1, k = N + i;
        const float sg = (i & 1) ? -1.0f : 1.0f;
        const float n0 = ax == 0 ? sg : 0.0f, n1 = ax == 1 ? sg : 0.0f, n2 = ax == 2 ? sg : 0.0f;
        if (M == kFP64) {
            double *r = s.r64 + 4 * k;
            r[0] = n0; r[1] = n1; r[2] = n2; r[3] = -a.box;
        } else {
            *reinterpret_cast<float4 *>(s.rhi + 4 * k) = make_float4(n0, n1, n2, -a.box_hi);
            *reinterpret_cast<float4 *>(s.rlo + 4 * k) = make_float4(0.0f, 0.0f, 0.0f, -a.box_lo);
            s.err[k] = 0.0f;
        }
    }
    if (tid == 0) {
        // an FP32 frame is enough: the square only has to contain the box section, and its
        // planes never bound a face (the box planes always cut them away)
        const float F[4] = {(float)s.aF[0], (float)s.aF[1], (float)s.aF[2], (float)s.aF[3]};
        const float nn = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
        int m = 0;
        if (nn > 0.0f && isfinite(nn)) {
            const float inn = 1.0f / nn;
            const float p0[3] = {-F[3] * F[0] * inn, -F[3] * F[1] * inn, -F[3] * F[2] * inn};
            const float inv = rsqrtf(nn);
            const float n[3] = {F[0] * inv, F[1] * inv, F[2] * inv};
            const float ax = fabsf(n[0]), ay = fabsf(n[1]), az = fabsf(n[2]);
            const int ei = (ax <= ay && ax <= az) ? 0 : (ay <= az ? 1 : 2);
            const float e0 = ei == 0 ? 1.0f : 0.0f, e1 = ei == 1 ? 1.0f : 0.0f, e2 = ei == 2 ? 1.0f : 0.0f;
            float u[3] = {n[1] * e2 - n[2] * e1, n[2] * e0 - n[0] * e2, n[0] * e1 - n[1] * e0};
            const float un = rsqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            u[0] *= un; u[1] *= un; u[2] *= un;
            const float w[3] = {n[1] * u[2] - n[2] * u[1], n[2] * u[0] - n[0] * u[2], n[0] * u[1] - n[1] * u[0]};
            const float sz = 1.05f * 1.7320508f * (float)a.box;
            // square edges -w, +u, +w, -u (ids N+6..N+9), counter-clockwise about n
            const float d[4][3] = {{-w[0], -w[1], -w[2]}, {u[0], u[1], u[2]}, {w[0], w[1], w[2]}, {-u[0], -u[1], -u[2]}};
            const float cu[4] = {-1.0f, 1.0f, 1.0f, -1.0f}, cw[4] = {-1.0f, -1.0f, 1.0f, 1.0f};
            for (int i = 0; i < 4; ++i) {
                const int k = N + kBoxPlanes + i;
                const float r[4] = {d[i][0], d[i][1], d[i][2], -(d[i][0] * p0[0] + d[i][1] * p0[1] + d[i][2] * p0[2]) - sz};
                for (int c = 0; c < 4; ++c) {
                    if (M == kFP64) s.r64[4 * k + c] = (double)r[c];
                    else { s.rhi[4 * k + c] = r[c]; s.rlo[4 * k + c] = 0.0f; }
                }
                if (M == kDF) s.err[k] = 0.0f;
                for (int c = 0; c < 3; ++c) {
                    const float x = p0[c] + sz * (cu[i] * u[c] + cw[i] * w[c]);
                    s.pv[0][i][c] = (double)x;
                    s.pf[0][i][c] = x;
                }
                s.pe[0][i] = k;
            }
            m = 4;
        }
        s.si[0] = m; s.si[1] = 0; s.si[2] = 0; s.si[3] = 0; s.si[4] = 0; s.si[5] = 0; s.si[9] = 0; s.si[10] = 0;
    }
    __syncthreads();
    // inverse norms, FP32 (they only scale distances used for ordering and the FP64 tolerance
    // test, never a sign)
    for (int k = tid; k < NC + kSquarePlanes; k += kT) {
        float n2;
        if (M == kFP64) {
            const double *r = s.r64 + 4 * k;
            n2 = (float)(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        } else {
            const float *r = s.rhi + 4 * k;
            n2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        }
        s.rinv[k] = n2 > 0.0f ? rsqrtf(n2) : 0.0f;
    }
    if (M == kDF) {
        // When a row's certified error, as a distance, exceeds kDfLoose the sign tests of this
        // cell cannot be certified in any useful number: the rigorous bound grows by the row
        // sums of |W_l| per layer (deep, wide nets).  Go to FP64 at once instead of clipping
        // twice.
        int loose = 0;
        for (int k = tid; k < N; k += kT) loose |= s.err[k] * s.rinv[k] > kDfLoose;
        if (tid == 0) loose |= s.eF[0] * rsqrtf((float)(s.aF[0] * s.aF[0] + s.aF[1] * s.aF[1] + s.aF[2] * s.aF[2])) > kDfLoose;
        if (__syncthreads_or(loose)) return CellOut{0, 1};
    } else {
        __syncthreads();
    }

    // ---- candidate rows, each thread keeps its best two, each warp contributes its four best:
    //      the rows nearest to the entry point, or the rows the learned proposal scores highest
    //      (the entry plane first), or none at all (the all-row check then clips alone)
    const bool learned = a.candidates == kCandLearned && a.prop.n_out == N && a.prop.n_in == 7 + net.L;
    float *score = (float *)s.viol;
    // the scores of a level batch come from the tensor cores; else this block computes them
    const __nv_bfloat16 *gscore = learned && a.scores_in ? a.scores_in + (cell - a.begin) * (int64_t)a.scores_ld : nullptr;
    if (learned && !gscore) proposal_scores(a, net, cell, s, score);
    {
        const float px = __ldcg(ar.entry_pt + cell * 3), py = __ldcg(ar.entry_pt + cell * 3 + 1),
                    pz = __ldcg(ar.entry_pt + cell * 3 + 2);
        const int entry = __ldcg(ar.entry_plane + cell);
        float b1 = 3.0e38f, b2 = 3.0e38f;
        int k1 = -1, k2 = -1;
        for (int k = (a.candidates == kCandNone ? NC : tid); k < NC; k += kT) {
            if (s.rinv[k] == 0.0f) continue;
            float d;
            if (learned) {
                if (k >= N) continue;
                d = k == entry ? -3.0e37f : -(gscore ? __bfloat162float(gscore[k]) : score[k]);
            } else if (M == kFP64) {
                const double *r = s.r64 + 4 * k;
                d = (float)fabs(r[0] * px + r[1] * py + r[2] * pz + r[3]) * s.rinv[k];
            } else {
                const float *r = s.rhi + 4 * k;
                d = fabsf(r[0] * px + r[1] * py + r[2] * pz + r[3]) * s.rinv[k];
            }
            if (d < b1) { b2 = b1; k2 = k1; b1 = d; k1 = k; }
            else if (d < b2) { b2 = d; k2 = k; }
        }
#pragma unroll 1
        for (int pick = 0; pick < kPicks; ++pick) {
            float bd = b1;
            int bk = k1;
            for (int o = 16; o > 0; o >>= 1) {
                const float od = __shfl_xor_sync(0xffffffffu, bd, o);
                const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
                if (ok >= 0 && (bk < 0 || od < bd || (od == bd && ok < bk))) { bd = od; bk = ok; }
            }
            if (lane == 0) { s.near_w[wid * kPicks + pick] = bk; s.near_dw[wid * kPicks + pick] = bd; }
            if (bk >= 0 && bk == k1) { b1 = b2; k1 = k2; b2 = 3.0e38f; k2 = -1; }
        }
    }
    __syncthreads();

    AM_TICK(tp2);
    // ---- a4: warp 0 cuts the square with the candidates, nearest cutting row first.  A row
    // that holds on the polygon holds on every later (smaller) one, so it retires at once.
    if (wid == 0) {
        float d = s.near_dw[lane];
        const int k = s.near_w[lane];
        bool live = k >= 0 && d < 3.0e38f;
        if (learned && live) {
            // the proposal chose the rows; they are cut nearest first, as the geometric rule's
            // (the entry plane passes through the entry point, so it still comes first)
            const float px = __ldcg(ar.entry_pt + cell * 3), py = __ldcg(ar.entry_pt + cell * 3 + 1),
                        pz = __ldcg(ar.entry_pt + cell * 3 + 2);
            float r[4];
            if (M == kFP64) {
                double r64[4];
                fetch_row<double, M>(s, k, r64);
                r[0] = (float)r64[0]; r[1] = (float)r64[1]; r[2] = (float)r64[2]; r[3] = (float)r64[3];
            } else {
                fetch_row<float, M>(s, k, r);
            }
            d = fabsf(r[0] * px + r[1] * py + r[2] * pz + r[3]) * s.rinv[k];
        }
        // order-preserving unsigned image of the distance (scores may be negative)
        const unsigned du = __float_as_uint(d);
        const unsigned key = (du & 0x80000000u) ? ~du : (du | 0x80000000u);
        AM_TICK(tp2a);
        int m = s.si[0], buf = 0, status = 0, ncut = 0;
        const float aFf[4] = {s.aFhi[0], s.aFhi[1], s.aFhi[2], s.aFhi[3]};
        while (m > 0) {
            bool cut = false;
            if (live) {
                if (M == kFP64) {
                    double r[4];
                    fetch_row<double, M>(s, k, r);
                    const double ri = (double)s.rinv[k];
                    for (int i = 0; i < m && !cut; ++i) cut = pdist(r, ri, s.pv[buf][i]) > a.delta;
                } else {
                    float r[4];
                    fetch_row<float, M>(s, k, r);
                    const float ri = s.rinv[k];
                    for (int i = 0; i < m && !cut; ++i) cut = pdist(r, ri, s.pf[buf][i]) > 1e-7f;
                }
            }
            live = cut;
            if (!__any_sync(0xffffffffu, cut)) break;
            const unsigned kmin = __reduce_min_sync(0xffffffffu, cut ? key : 0xffffffffu);
            const int kc = (int)__reduce_min_sync(0xffffffffu, (cut && key == kmin) ? (unsigned)k : 0xffffffffu);
            if (k == kc) live = false;
            bool sw;
            int nm;
            if (M == kFP64) nm = warp_cut<double, M>(s, s.pv, m, buf, kc, a.delta, s.aF, &sw);
            else nm = warp_cut<float, M>(s, s.pf, m, buf, kc, 1e-7f, aFf, &sw);
            if (nm < 0) { status = 1; m = 0; break; }
            if (sw) buf ^= 1;
            m = nm;
            ++ncut;
        }
        AM_TICK(tp3a);
        if (M == kDF && m > 0) df_final_vertices(s, m, buf, kVertexTol);
        if (lane == 0) { s.si[0] = m; s.si[1] = buf; s.si[2] = status; s.blk[6] += (unsigned long long)ncut; }
    }
    __syncthreads();

    AM_TICK(tp3);
    // ---- a5: every row at every vertex; violators are cut in by warp 0 and the check repeats
    int rounds = 0;
    for (;; ++rounds) {
        const int m = s.si[0], buf = s.si[1];
        if (M == kDF && s.si[10]) return CellOut{0, 1};     // a vertex too uncertain: FP64
        // kDF: a polygon emptied (or a clip that failed) in the uncertified FP32 candidate pass
        // proves nothing: FP64 decides
        if (M == kDF && (m == 0 || s.si[2])) return CellOut{0, 1};
        if (m == 0 || s.si[2]) break;
        for (int i = tid; i < m; i += kT) {
            const double *v = s.pv[buf][i];
            s.vf[i][0] = (float)v[0]; s.vf[i][1] = (float)v[1]; s.vf[i][2] = (float)v[2];
            s.vf[i][3] = (float)fmax(1.0, fmax(fabs(v[0]), fmax(fabs(v[1]), fabs(v[2])))) * 1.0001f;
        }
        if (tid == 0) { s.si[3] = 0; s.si[4] = 0; }
        __syncthreads();
        int ndeg = 0, close = 0;
        for (int k = tid; k < NC; k += kT) {
            if (s.rinv[k] == 0.0f) continue;        // zero normal: constant row, holds in its own cell
            bool viol = false, amb = false;
            if (M == kFP64) {
                const double *r = s.r64 + 4 * k;
                const double ri = (double)s.rinv[k];
                for (int i = 0; i < m; ++i) {
                    const int ea = s.pe[buf][(i + m - 1) % m], eb = s.pe[buf][i];
                    if (k == ea || k == eb) continue;
                    const double dd = pdist(r, ri, s.pv[buf][i]);
                    if (dd > a.delta) viol = true;
                    else if (dd >= -a.delta) ++ndeg;
                }
            } else {
                const float *r = s.rhi + 4 * k;
                const float rl1 = fabsf(r[0]) + fabsf(r[1]) + fabsf(r[2]);
                const float band = (float)a.delta / s.rinv[k] * 1.01f;   // delta |r|: the oracle's tolerance band
                const float ek = s.err[k];
                for (int i = 0; i < m; ++i) {
                    const int ea = s.pe[buf][(i + m - 1) % m], eb = s.pe[buf][i];
                    if (k == ea || k == eb) continue;
                    const float *v = s.vf[i];
                    const float sl = r[0] * v[0] + r[1] * v[1] + r[2] * v[2] + r[3];
                    const float mag = fabsf(r[0] * v[0]) + fabsf(r[1] * v[1]) + fabsf(r[2] * v[2]) + fabsf(r[3]);
                    // FP32 evaluation (4 terms) + dropping lo + rounding v to FP32: (4 + 4) u |r||v|
                    const float B = __fmaf_ru(8.5f * kU, mag, __fmaf_ru(ek, v[3], __fmaf_ru(rl1, s.dvb[i], band)));
                    if (sl > B) { viol = true; continue; }
                    if (sl >= -B) {                    // close call: FP64 re-evaluation
                        ++close;
                        double r6[4];
                        row64<kDF>(s, k, r6);
                        const double *v6 = s.pv[buf][i];
                        const double s6 = r6[0] * v6[0] + r6[1] * v6[1] + r6[2] * v6[2] + r6[3];
                        const double m6 = fabs(r6[0] * v6[0]) + fabs(r6[1] * v6[1]) + fabs(r6[2] * v6[2]) + fabs(r6[3]);
                        const double B6 = (double)ek * (double)v[3] + (double)rl1 * 1.0001 * (double)s.dvb[i] +
                                          (double)band + 1e-15 * m6;
                        if (s6 > B6) viol = true;
                        else if (s6 >= -B6) amb = true;
                    }
                }
                // A violated row that already carries an edge of the polygon: the FP32 candidate
                // pass cut by a row that does not really cut the face (its exact vertices then lie
                // outside the neighbouring edges' rows).  Cutting again would repeat that plane
                // with a zero-length edge, so the cell goes to FP64, which decides every cut.
                if (viol)
                    for (int i = 0; i < m; ++i) amb |= s.pe[buf][i] == k;
            }
            if (viol) {
                const int p = atomicAdd(s.si + 3, 1);
                s.viol[p] = k;
            }
            if (amb) s.si[4] = 1;
        }
        {
            int tot;
            block_scan_excl(ndeg, s.wsum, &tot);
            ndeg = tot;
            block_scan_excl(close, s.wsum, &tot);
            if (tid == 0) s.blk[5] += (unsigned long long)tot;
        }
        if (tid == 0) s.si[5] = ndeg;
        __syncthreads();
        if (s.si[4]) return CellOut{0, 1};
        const int nviol = s.si[3];
        if (nviol == 0) break;
        if (rounds + 1 >= kMaxFix) {
            if (tid == 0) s.si[2] = 2;
            __syncthreads();
            break;
        }
        if (wid == 0) {
            int mm = m, bb = buf, status = 0, t = 0;
            const double tol = M == kFP64 ? a.delta : 0.0;
            bool changed = false;
            for (; t < nviol && mm > 0; ++t) {
                bool sw;
                const int nm = warp_cut<double, M>(s, s.pv, mm, bb, s.viol[t], tol, s.aF, &sw);
                if (nm < 0) { status = 1; mm = 0; break; }
                if (sw) bb ^= 1;
                changed |= sw || nm != mm;
                mm = nm;
            }
            if (M == kDF && mm > 0) df_final_vertices(s, mm, bb, kVertexTol);
            if (lane == 0) {
                s.si[0] = mm; s.si[1] = bb; s.si[2] = status; s.si[9] += 1; s.blk[6] += (unsigned long long)t;
                // kDF: rows the certified FP32 test calls violated that the cut on the pairs in FP64
                // does not move: the two views of the rows disagree, so FP64 decides the cell
                if (M == kDF && !changed && status == 0) s.si[10] = 1;
            }
        }
        __syncthreads();
    }

    AM_TICK(tp4);
    // ---- a6 emit, a7 march
    const int m = s.si[0], buf = s.si[1];
    int status = s.si[2];
    for (int i = 0; i < m; ++i)
        if (s.pe[buf][i] >= N + kBoxPlanes) status = 3;   // a square edge: the plane misses the box
    int emit = (m >= 3 && status == 0) ? m : 0;
    if (emit && wid == 0) {
        // area of the polygon, as a fan about vertex 0 summed over the warp's lanes
        const double *p0 = s.pv[buf][0];
        double nx = 0.0, ny = 0.0, nz = 0.0;
        for (int i = lane + 1; i < m - 1; i += 32) {
            const double *p = s.pv[buf][i], *q = s.pv[buf][i + 1];
            const double ax = p[0] - p0[0], ay = p[1] - p0[1], az = p[2] - p0[2];
            const double bx = q[0] - p0[0], by = q[1] - p0[1], bz = q[2] - p0[2];
            nx += ay * bz - az * by; ny += az * bx - ax * bz; nz += ax * by - ay * bx;
        }
        nx = warp_sum(nx); ny = warp_sum(ny); nz = warp_sum(nz);
        const double amin = 2e-24 * a.box * a.box;          // twice the smallest kept area
        if (lane == 0) s.si[6] = nx * nx + ny * ny + nz * nz > amin * amin;
    }
    __syncthreads();
    if (emit && !s.si[6]) emit = 0;
    if (emit > ar.maxv) {
        if (tid == 0) atomicOr(ar.counters + kStatus, kStFaceVerts);
        emit = 0;
    }
    if (tid == 0) {
        ar.nverts[cell] = emit;
        s.blk[0] += 1;
        if (!emit) s.blk[1] += 1;
        if (emit) s.blk[2] += (unsigned long long)s.si[5];
        if (rounds) s.blk[3] += 1;
        if (status == 1 || status == 2) atomicOr(ar.counters + kStatus, kStClip);
    }
    AM_TICK(tp4a);
    if (emit) {
        for (int i = tid; i < m; i += kT) {
            ar.edges[cell * ar.maxv + i] = s.pe[buf][i];
            double *v = ar.verts + (cell * ar.maxv + i) * 3;
            v[0] = s.pv[buf][i][0]; v[1] = s.pv[buf][i][1]; v[2] = s.pv[buf][i][2];
        }
        const unsigned long long h = __ldcg(ar.hash + cell);
        const int nid = __ldcg(ar.net + cell);
        // a max-pooled net (Sec. 5.2): crossing pooling plane n_units + i moves the pooled index j
        // to i (two key bits change), and the new cell enters through its pooling row of j
        int pj = 0;
        if (net.M >= 2)
            for (int i = 0; i < net.M; ++i)
                if (bit_of(s.mask, net.n_units + i)) { pj = i; break; }
        const int pool0 = net.M >= 2 ? net.n_units : kNoPool, pool1 = net.M >= 2 ? N : kNoPool;
        auto child = [&](int e, unsigned long long *hc, int *entry) {
            if (e >= pool0 && e < pool1) {
                *hc = h ^ ar.zob[e] ^ ar.zob[pool0 + pj];
                *entry = pool0 + pj;
            } else {
                *hc = h ^ ar.zob[e];
                *entry = -1;
            }
        };
        if (ar.kw <= kThreadPushWords) {
            // narrow keys: one thread per edge
            for (int i = tid; i < m; i += kT) {
                const int e = s.pe[buf][i];
                if (e >= N) continue;
                const double *p = s.pv[buf][i], *q = s.pv[buf][(i + 1) % m];
                unsigned long long hc;
                int entry;
                child(e, &hc, &entry);
                insert_neighbor(ar, s.mask, cell, nid, (unsigned)e, hc, (float)(0.5 * (p[0] + q[0])),
                                (float)(0.5 * (p[1] + q[1])), (float)(0.5 * (p[2] + q[2])), pool0, pool1, entry);
            }
        } else {
            // wide keys: one warp per edge, the key words split over the lanes
            for (int i = wid; i < m; i += kNW) {
                const int e = s.pe[buf][i];
                if (e >= N) continue;
                const double *p = s.pv[buf][i], *q = s.pv[buf][(i + 1) % m];
                unsigned long long hc;
                int entry;
                child(e, &hc, &entry);
                insert_neighbor_warp(ar, s.mask, cell, nid, (unsigned)e, hc, (float)(0.5 * (p[0] + q[0])),
                                     (float)(0.5 * (p[1] + q[1])), (float)(0.5 * (p[2] + q[2])), true, pool0,
                                     pool1, entry);
            }
        }
    }
    if (emit && tid < m) __threadfence();     // the face and the pushes of this thread
    __syncthreads();
    AM_TICK(tp5);
    AM_PHASE(a, 0, tp0, tp1);
    AM_PHASE(a, 1, tp1, tp2);
    AM_PHASE(a, 2, tp2, tp2a);
    AM_PHASE(a, 3, tp2a, tp3a);
    AM_PHASE(a, 4, tp3a, tp3);
    AM_PHASE(a, 5, tp3, tp4);
    AM_PHASE(a, 6, tp4, tp4a);
    AM_PHASE(a, 7, tp4a, tp5);
    return CellOut{emit, 0};
}

template <int MODE>
__device__ void process_cell(const MarchArgs &a, int64_t cell, const Sh &s)
{
    const Arena &ar = a.ar;
    // the cell's record was written by another block of this launch: read it through L2
    if (__ldcg(ar.nverts + cell) == -2) return;          // a duplicate seed id: never solved
    const NetDev &net = a.nets[__ldcg(ar.net + cell)];
    const unsigned long long *key = ar.keys + cell * ar.kw;
    for (int w = threadIdx.x; w < 2 * ar.kw; w += kT)       // all key words: pushes copy them
        s.mask[w] = (unsigned)(__ldcg(key + (w >> 1)) >> ((w & 1) * 32));
    __syncthreads();
    if (MODE == kDF && !net.df_ok && !a.rows_in) {
        if (threadIdx.x == 0) s.blk[4] += 1;             // solved in FP64 (the net's bound is too loose)
        solve_cell<kFP64>(a, net, cell, s);
    } else if (MODE == kDF) {
        const CellOut o = solve_cell<kDF>(a, net, cell, s);
        if (o.ambiguous) {
            if (threadIdx.x == 0) s.blk[4] += 1;
            solve_cell<kFP64>(a, net, cell, s);
        }
    } else {
        solve_cell<kFP64>(a, net, cell, s);
    }
}

// ------------------------------------------------------------------------------------------
// schedules

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Ticket of the next cell to solve, or -1 when the march is over (every handed-out cell is
// finished), the ticket is beyond the limit, or a wait ran out of time (status flag set).
// Waiting polls with plain acquire loads and an exponential back-off, so that idle blocks do
// not flood the counters' cache lines with atomics.
__device__ long long next_ticket(const MarchArgs &a)
{
    unsigned long long *C = a.ar.counters;
    const long long t = (long long)atomicAdd(C + kHead, 1ull);
    if (t >= a.limit) return -1;
    const long long t0 = global_ns();
    unsigned ns = 32;
    for (;;) {
        const unsigned long long n = ld_acquire(C + kNCells);
        if ((unsigned long long)t < n) {
            unsigned ns2 = 16;
            while (ld_acquire(a.ar.ready + t) == 0u) {
                if (global_ns() - t0 > a.wait_ns) { atomicOr(C + kStatus, kStTimeout); return -1; }
                __nanosleep(ns2);
                ns2 = min(2 * ns2, 256u);
            }
            return t;
        }
        // every handed-out cell finished (done read before the count: no cell can still push)
        const unsigned long long done = ld_acquire(C + kDone);
        const unsigned long long n2 = ld_acquire(C + kNCells);
        if (done >= n2 && (unsigned long long)t >= n2) return -1;
        if (global_ns() - t0 > a.wait_ns) { atomicOr(C + kStatus, kStTimeout); return -1; }
        __nanosleep(ns);
        ns = min(2 * ns, 256u);
    }
}

// per-block statistics: zero at entry, one atomic flush at exit
__device__ __forceinline__ void blk_init(const Sh &s)
{
    if (threadIdx.x < 8) s.blk[threadIdx.x] = 0ull;
    __syncthreads();
}

__device__ __forceinline__ void blk_flush(const MarchArgs &a, const Sh &s)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long *C = a.ar.counters;
        if (s.blk[0]) atomicAdd(C + kSolved, s.blk[0]);
        if (s.blk[1]) atomicAdd(C + kEmpty, s.blk[1]);
        if (s.blk[2]) atomicAdd(C + kDegenerate, s.blk[2]);
        if (s.blk[3]) atomicAdd(C + kFixups, s.blk[3]);
        if (s.blk[4]) atomicAdd(C + kRefined, s.blk[4]);
        if (s.blk[5]) atomicAdd(C + kCloseCalls, s.blk[5]);
        if (s.blk[6]) atomicAdd(C + kCuts, s.blk[6]);
    }
}

template <int MODE>
__global__ void __launch_bounds__(kT, AM_MIN_BLOCKS) march_persistent_kernel(MarchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Sh s = make_sh(smem, a.max_n, a.max_w);
    __shared__ long long ticket;
    blk_init(s);
    for (;;) {
        long long tw0 = 0, tw1 = 0;
        AM_TICK(tw0);
        if (threadIdx.x == 0) ticket = next_ticket(a);
        __syncthreads();
        AM_TICK(tw1);
        AM_PHASE(a, 8, tw0, tw1);
        const long long t = ticket;
        if (t < 0) break;
        process_cell<MODE>(a, t, s);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(a.ar.counters + kDone, 1ull);
        }
    }
    blk_flush(a, s);
}

template <int MODE>
__global__ void __launch_bounds__(kT, AM_MIN_BLOCKS) march_range_kernel(MarchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Sh s = make_sh(smem, a.max_n, a.max_w);
    blk_init(s);
    if (a.list) {
        const int64_t n = (int64_t)__ldcg(a.list_count);
        for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
            process_cell<MODE>(a, a.list[i], s);
            __syncthreads();
        }
    } else {
        for (int64_t cell = a.begin + blockIdx.x; cell < a.end; cell += gridDim.x) {
            process_cell<MODE>(a, cell, s);
            __syncthreads();
        }
    }
    blk_flush(a, s);
}

template <int MODE>
__global__ void __launch_bounds__(kT, AM_MIN_BLOCKS)
    compose_kernel(MarchArgs a, const NetDev *netp, const unsigned long long *keys, int kw_in, int64_t n,
                   double *rows, float *err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Sh s = make_sh(smem, a.max_n, a.max_w);
    const NetDev &net = *netp;
    const int N = net.N, mw = 2 * ((a.max_n + 63) / 64);
    for (int64_t c = blockIdx.x; c < n; c += gridDim.x) {
        for (int w = threadIdx.x; w < mw; w += kT)
            s.mask[w] = (w >> 1) < kw_in ? (unsigned)(keys[c * kw_in + (w >> 1)] >> ((w & 1) * 32)) : 0u;
        __syncthreads();
        compose<MODE>(net, s, a.tc != 0, a.max_n + kBoxPlanes + kSquarePlanes);
        double *out = rows + c * (int64_t)(N + 1) * 4;
        for (int k = threadIdx.x; k < N; k += kT) {
            double r[4];
            row64<MODE>(s, k, r);
            out[4 * k] = r[0]; out[4 * k + 1] = r[1]; out[4 * k + 2] = r[2]; out[4 * k + 3] = r[3];
            if (err) err[c * (N + 1) + k] = MODE == kFP64 ? 0.0f : s.err[k];
        }
        if (threadIdx.x == 0) {
            for (int q = 0; q < 4; ++q) out[4 * N + q] = s.aF[q];
            if (err) err[c * (N + 1) + N] = MODE == kFP64 ? 0.0f : s.eF[0];
        }
        __syncthreads();
    }
}

void launch_compose(const MarchArgs &a, int mode, const NetDev *net, const unsigned long long *keys, int key_words,
                    int64_t n, double *rows, float *err, cudaStream_t st)
{
    const int smem = march_smem_bytes(a.max_n, a.max_w);
    const int grid = (int)std::min<int64_t>(n, 152 * 8);
    if (mode == kDF) compose_kernel<kDF><<<grid, kT, smem, st>>>(a, net, keys, key_words, n, rows, err);
    else compose_kernel<kFP64><<<grid, kT, smem, st>>>(a, net, keys, key_words, n, rows, err);
}

cudaError_t prepare_march_kernels(int max_n, int max_w, int *blocks_per_sm)
{
    const int smem = march_smem_bytes(max_n, max_w);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(march_persistent_kernel<kFP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    if ((e = cudaFuncSetAttribute(march_persistent_kernel<kDF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    if ((e = cudaFuncSetAttribute(march_range_kernel<kFP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    if ((e = cudaFuncSetAttribute(march_range_kernel<kDF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    if ((e = cudaFuncSetAttribute(compose_kernel<kFP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    if ((e = cudaFuncSetAttribute(compose_kernel<kDF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    // shared memory for two resident blocks, the rest of the unified L1 for the weights and
    // the stack (the driver rounds the carveout to a supported split)
    const int carve = std::min(100, (int)((2.0 * (smem + 1024) * 100.0) / (228.0 * 1024.0)) + 3);
    const void *ks[4] = {(const void *)march_persistent_kernel<kFP64>, (const void *)march_persistent_kernel<kDF>,
                         (const void *)march_range_kernel<kFP64>, (const void *)march_range_kernel<kDF>};
    for (const void *k : ks)
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
    int b0 = 0, b1 = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, march_persistent_kernel<kFP64>, kT, smem))) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, march_persistent_kernel<kDF>, kT, smem))) return e;
    *blocks_per_sm = b0 < b1 ? b0 : b1;
    return cudaSuccess;
}

void launch_march(const MarchArgs &a, int mode, bool persistent, int grid, cudaStream_t st)
{
    const int smem = march_smem_bytes(a.max_n, a.max_w);
    if (persistent) {
        if (mode == kDF) march_persistent_kernel<kDF><<<grid, kT, smem, st>>>(a);
        else march_persistent_kernel<kFP64><<<grid, kT, smem, st>>>(a);
    } else {
        if (mode == kDF) march_range_kernel<kDF><<<grid, kT, smem, st>>>(a);
        else march_range_kernel<kFP64><<<grid, kT, smem, st>>>(a);
    }
}

}  // namespace am
