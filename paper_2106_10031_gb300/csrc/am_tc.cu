// am_tc.cu -- the compose step (Lemma 1, Cor. 1) on the tcgen05 tensor cores, with the
// activation patterns of K cells stacked as the columns of one right operand.
//
// Per hidden layer l >= 2 the compose is the product Z_l = W_l diag(s_{l-1}) Z_{l-1} + C_l, and
// for a batch of cells the right operands diag(s_{l-1}) Z_{l-1} (4 columns per cell) stack into
// one [n_{l-1} x 4K] matrix: one dense contraction per layer for the whole batch.
//
// Error-free slicing (Ozaki, Ogita, Oishi & Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its applications",
// Numer. Algorithms 59, 2012).  Every row m of W_l is written as
//     W_m = 2^eA_m sum_{s=1..8} a_s 2^(-6 s),   integers |a_1| <= 64, |a_s| <= 32 (s >= 2),
// and every column c of the stacked operand likewise with its own exponent eB_c.  The digits
// are integers that BF16 holds exactly, so the product of two digit planes is exact, and the
// tensor core's FP32 accumulator only ever adds integers whose running sum stays below 2^24
// (n_{l-1} <= 1638), which is exact too.  The products of the planes (s, t) with the same
// diagonal s + t share one scale and accumulate into one TMEM accumulator (36 plane products
// over 8 diagonals).  The epilogue combines the diagonals exactly in 64-bit integers; the prep
// kernel converts once to FP64 (or to FP32 pairs for the march).  What is dropped are the
// planes with s + t > 9 and the residuals after 8 digits: per output at most
// (3 n_{l-1} + 1) 2^-48 2^(eA_m + eB_c), the same order as the worst-case rounding of an FP64
// dot product of that length.  So the rows are FP64-class, and the march can clip them with
// the tests it uses for FP64 rows.
//
// Kernels (per layer and batch):
//   oz_prep_kernel      : the rows of layer l from the exact products (exponents, C_l, the sign
//                         (1 - 2 s_k) of Eq. 10; layer 1 is cell independent), then, per cell
//                         and coordinate, the column exponent and the 8 BF16 digit planes of
//                         diag(s_l) Z_l for the next layer (integer arithmetic on the bit
//                         patterns), or, after the last layer, a_F = w_out^T diag(s_L) Z_L +
//                         [0 | b_out] (Eq. 8);
//   oz_gemm_kernel      : one CTA per 128 rows of W_l x NC cells (NC = 16 or 8).  Warp 0 stages
//                         digit-plane tiles of W_l and of the stacked operand into shared memory
//                         with TMA (128-byte swizzle), warp 1 issues tcgen05.mma (M = 128,
//                         N = 4 NC, K = 16) into 8 TMEM accumulators, keeping each A slice in
//                         the collector, warps 2..5 read them back with tcgen05.ld and write
//                         the exact products as 64-bit integers;
//   oz_gemm_wide_kernel : the same for 32 cells (N = 128), the diagonals in two passes of 4.
// Every wait on an mbarrier has a time limit; when one runs out the kernel raises a flag the
// host reads, lets its copies and products in flight finish, frees its TMEM and returns.
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <cmath>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <vector>

#include "am_kernels.h"
#include "am_tcgen05.cuh"

namespace am {

namespace {

using namespace tc;

constexpr int kOzPlanes = kOzDigits;      // digit planes per operand = accumulator diagonals
constexpr int kOzBK = 64;                 // K elements per staged chunk (128 bytes of BF16)
constexpr int kOzM = 128;                 // rows of W_l per CTA (UMMA M)
constexpr int kOzPrepThreads = 128;       // threads of the prep block of one cell
constexpr long long kOzDrainNs = kDrainNs;     // limit on the drain after an abort

// acc 2^e as a double, rounded to nearest even, with integer operations on the bit pattern
// (the FP64 pipe of this part is narrow); results outside the normal range go through ldexp
__device__ __forceinline__ double i64_ldexp(long long acc, int e)
{
    if (acc == 0) return 0.0;
    const unsigned long long sgn = acc < 0 ? 0x8000000000000000ull : 0ull;
    unsigned long long m = acc < 0 ? 0ull - (unsigned long long)acc : (unsigned long long)acc;
    const int sh = 11 - __clzll(m);               // bits beyond 53
    if (sh > 0) {
        const unsigned long long rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        m >>= sh;
        if (rem > half || (rem == half && (m & 1ull))) ++m;
        e += sh;
        if (m >> 53) { m >>= 1; ++e; }
    } else {
        m <<= -sh;
        e += sh;
    }
    const int be = e + 52 + 1023;                 // m in [2^52, 2^53)
    if (be <= 0 || be >= 2047) return ldexp(sgn ? -(double)m : (double)m, e);
    return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ bool key_bit(const unsigned long long *key, int k) { return (key[k >> 6] >> (k & 63)) & 1ull; }

// Exponent e with |x| <= 2^e for every x of a column whose largest |x| has the bit pattern
// `mx` (sign cleared); 0 for an all-zero column.
__device__ __forceinline__ int col_exponent(unsigned long long mx)
{
    if (mx == 0ull) return 0;
    const int be = (int)(mx >> 52);
    if (be == 0) return -1022;                                  // subnormal maximum
    return be - 1023 + ((mx & 0xFFFFFFFFFFFFFull) != 0ull ? 1 : 0);
}

// x = z 2^(62 - e) as a 64-bit integer (|z| <= 2^e, so |x| <= 2^62), the bits of z below
// 2^(e - 62) truncated; integer operations on the bit pattern only.
__device__ __forceinline__ long long fixed62(double z, int e)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(z);
    const int be = (int)((u >> 52) & 0x7FF);
    if (be == 0) return 0;                                      // zero or subnormal: below 2^-1022
    const long long mant = (long long)((u & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
    const int sh = be - 1013 - e;                               // mant 2^(be-1075) * 2^(62-e)
    long long x;
    if (sh >= 0) x = mant << sh;                                // sh <= 10 since |z| <= 2^e
    else if (sh > -64) x = mant >> (-sh);
    else x = 0;
    return (u >> 63) ? -x : x;
}

// BF16 bits of a small integer d (|d| <= 64), exact
__device__ __forceinline__ unsigned bf16_of_int(int d) { return __float_as_uint((float)d) >> 16; }

// ------------------------------------------------------------------------------------------
// digit planes of the stacked operand, layer-1 rows, a_F

struct OzPrep {
    const unsigned long long *keys;   // cell i's key at keys + i * kw (list: at keys + list[i] * kw)
    const int32_t *list;              // null, or the cell ids of the batch (rows at rows + (list[i] - cell0) rstride)
    int64_t cell0;
    int kw;
    int64_t n;                        // cells in the batch
    void *rows;                       // cell i's rows at rows + i * rstride (N rows, then a_F), 32 B each:
    int64_t rstride;                  //   FP64 [a | a0], or, when df, FP32 pairs as two blocks: the N + 1
                                      //   hi words [hi x4] first, then the N + 1 lo words [lo x4]
    int df;
    int l, L, N;
    int nl, row0;                     // width and first neuron of layer l
    long long *P, *Q;                 // l >= 2: the exact products of layer l (diagonals 0..6, and the raw
                                      // sum of diagonal 7), column c at P + c Mp; zeroed once read when
    int zero;                         // zero is set (the product added split-K partial sums into them)
    int Mp;
    const int *eA;                    // l >= 2: row exponents of W_l
    const int *eBin;                  // l >= 2: column exponents of layer l's right operand
    const double *Cl;                 // layer l constant rows (n_l x 4), FP64 ...
    const float *Clhi, *Cllo;         // ... and as double-float pairs
    const double *w_out;
    double b_out;
    __nv_bfloat16 *B;                 // digit planes for layer l + 1: plane t, column c at row t ncols + c
    int *eBout;                       // column exponents for layer l + 1
    int64_t ncols;
    int Kp;                           // round_up(n_l, 64)
};

// (sh, sl) += (bh, bl): double-float addition, TwoSum on the high parts (Knuth), then the
// renormalisation |sl| <= ulp(sh) / 2 (Fast2Sum)
__device__ __forceinline__ void df_add(float &sh, float &sl, float bh, float bl)
{
    const float t = __fadd_rn(sh, bh);
    const float bp = __fsub_rn(t, sh);
    const float te = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(bh, bp));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(te, bl));
}

__device__ __forceinline__ void df_norm(float &h, float &l)
{
    const float s = __fadd_rn(h, l);
    l = __fsub_rn(l, __fsub_rn(s, h));
    h = s;
}

// nearest FP32 of acc 2^e (integer operations; outside the normal range through ldexpf) and the
// 64-bit integer that FP32 stands for at scale 2^e
__device__ __forceinline__ float i64_to_f32(long long acc, int e, long long *as_int)
{
    if (acc == 0) { *as_int = 0; return 0.0f; }
    const bool neg = acc < 0;
    unsigned long long m = neg ? 0ull - (unsigned long long)acc : (unsigned long long)acc;
    const int sh = 40 - __clzll(m);               // bits beyond 24
    int ee = e;
    if (sh > 0) {
        const unsigned long long rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        m >>= sh;
        if (rem > half || (rem == half && (m & 1ull))) ++m;
        ee += sh;
        *as_int = (long long)(m << sh);
        if (m >> 24) { m >>= 1; ++ee; }
    } else {
        *as_int = (long long)m;
        m <<= -sh;
        ee += sh;
    }
    if (neg) *as_int = -*as_int;
    const int be = ee + 23 + 127;                 // m in [2^23, 2^24)
    float f;
    if (be <= 0 || be >= 255) f = ldexpf((float)m, ee);
    else f = __uint_as_float(((unsigned)be << 23) | ((unsigned)m & 0x7FFFFFu));
    return neg ? -f : f;
}

// x 2^(62 - e) as a 64-bit integer for an FP32 x with |x| < 2^e (truncated below 2^(e - 62))
__device__ __forceinline__ long long fixed62f(float x, int e)
{
    const unsigned u = __float_as_uint(x);
    const int be = (int)((u >> 23) & 0xFF);
    if (be == 0) return 0;
    const long long mant = (long long)((u & 0x7FFFFFu) | 0x800000u);
    const int sh = be - 88 - e;                   // mant 2^(be-150) 2^(62-e)
    long long v;
    if (sh >= 0) v = mant << sh;
    else if (sh > -64) v = mant >> (-sh);
    else v = 0;
    return (u >> 31) ? -v : v;
}

// The exact product of column 4 i + j, row k at scale 2^-48: P (diagonals 0..6, or 0..3 for the
// wide tile) plus Q (diagonal 7, or diagonals 4..7 for the wide tile, at scale 2^-54) rounded to
// the scale once, after every split of K has added in (so the rows do not depend on the launch
// shape)
__device__ __forceinline__ long long oz_product(const OzPrep &p, int64_t i, int j, int k)
{
    const int64_t o = (4 * i + j) * p.Mp + k;
    const long long v = p.P[o] + ((p.Q[o] + 32) >> 6);
    if (p.zero) {                                 // consumed: zero for the next product's split-K sums
        p.P[o] = 0;
        p.Q[o] = 0;
    }
    return v;
}

// One block of kOzPrepThreads per cell: the rows of layer l (from the exact products, or the
// cell-independent C_1 at layer 1), then the digit planes of diag(s_l) Z_l for layer l + 1, or
// a_F after the last layer.
__global__ void __launch_bounds__(kOzPrepThreads) oz_prep_kernel(OzPrep p)
{
    constexpr int kW = kOzPrepThreads / 32;
    __shared__ unsigned long long red[kW][4];
    __shared__ double fred[kW][4];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t i = blockIdx.x;
    const int64_t cell = p.list ? (int64_t)p.list[i] : i;
    const unsigned long long *key = p.keys + cell * p.kw;
    double *out = reinterpret_cast<double *>(p.rows) + (p.list ? cell - p.cell0 : i) * p.rstride;   // 4 doubles = 8 floats per row
    float *outf = reinterpret_cast<float *>(out);
    // ---- rows of layer l, signed (1 - 2 s_k) as in Eq. 10, and the column maxima of
    //      |diag(s_l) Z_l| (bit patterns of non-negative values order as integers)
    unsigned long long mx[4] = {0ull, 0ull, 0ull, 0ull};
    for (int k = tid; k < p.nl; k += kOzPrepThreads) {
        const int r = p.row0 + k;
        const bool act = key_bit(key, r);
        if (!p.df) {
            double v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (p.l == 1) v[j] = p.Cl[4 * k + j];
                else v[j] = i64_ldexp(oz_product(p, i, j, k), p.eA[k] + p.eBin[4 * i + j] - 48) + p.Cl[4 * k + j];
                if (act) v[j] = -v[j];
                if (act) {
                    const unsigned long long a = (unsigned long long)__double_as_longlong(v[j]) & 0x7FFFFFFFFFFFFFFFull;
                    mx[j] = a > mx[j] ? a : mx[j];
                }
            }
            double2 *o = reinterpret_cast<double2 *>(out + 4 * (int64_t)r);
            o[0] = make_double2(v[0], v[1]);
            o[1] = make_double2(v[2], v[3]);
        } else {
            float h[4], lo[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                h[j] = p.Clhi[4 * k + j];
                lo[j] = p.Cllo[4 * k + j];
                if (p.l > 1) {
                    const long long acc = oz_product(p, i, j, k);
                    const int e = p.eA[k] + p.eBin[4 * i + j] - 48;
                    long long hi_int;
                    const float ah = i64_to_f32(acc, e, &hi_int);
                    long long lo_int;
                    const float al = i64_to_f32(acc - hi_int, e, &lo_int);
                    df_add(h[j], lo[j], ah, al);
                    df_norm(h[j], lo[j]);
                }
                if (act) {
                    h[j] = -h[j];
                    lo[j] = -lo[j];
                    const unsigned long long a = __float_as_uint(h[j]) & 0x7FFFFFFFu;
                    mx[j] = a > mx[j] ? a : mx[j];
                }
            }
            float4 *o = reinterpret_cast<float4 *>(outf);
            o[r] = make_float4(h[0], h[1], h[2], h[3]);
            o[p.N + 1 + r] = make_float4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
    __syncthreads();                               // the block reads back the rows it wrote
    const double *Z = out + 4 * (int64_t)p.row0;
    const float *Zh = outf + 4 * (int64_t)p.row0, *Zl = outf + 4 * (int64_t)(p.N + 1 + p.row0);   // df: the pairs
    if (p.l == p.L) {
        // a_F = w_out^T diag(s_L) Z_L + [0 | b_out] (Cor. 1, Eq. 8); an active row is -Z_k
        double f[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = tid; k < p.nl; k += kOzPrepThreads)
            if (key_bit(key, p.row0 + k)) {
                const double w = p.w_out[k];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const double r = p.df ? (double)Zh[4 * k + j] + (double)Zl[4 * k + j] : Z[4 * k + j];
                    f[j] = fma(-w, r, f[j]);
                }
            }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            for (int o = 16; o > 0; o >>= 1) f[j] += __shfl_xor_sync(0xffffffffu, f[j], o);
            if (lane == 0) fred[wid][j] = f[j];
        }
        __syncthreads();
        if (tid < 4) {
            double F = tid == 3 ? p.b_out : 0.0;
            for (int w = 0; w < kW; ++w) F += fred[w][tid];
            if (!p.df) {
                out[4 * (int64_t)p.N + tid] = F;
            } else {
                const float h = (float)F;
                outf[4 * (int64_t)p.N + tid] = h;
                outf[4 * (int64_t)(2 * p.N + 1) + tid] = (float)(F - (double)h);
            }
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx[j], o);
            mx[j] = v > mx[j] ? v : mx[j];
        }
        if (lane == 0) red[wid][j] = mx[j];
    }
    __syncthreads();
    int e[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        unsigned long long m = 0ull;
        for (int w = 0; w < kW; ++w) m = red[w][j] > m ? red[w][j] : m;
        if (!p.df) {
            e[j] = col_exponent(m);
        } else {
            // |hi + lo| <= |hi| (1 + 2^-24): one binade of headroom above the largest |hi|
            const int be = (int)(m >> 23);
            e[j] = m == 0ull ? 0 : (be == 0 ? -126 : be - 127 + 1);
        }
    }
    if (tid < 4) p.eBout[4 * i + tid] = e[tid];
    // digits: two consecutive k per thread, so each plane store is a BF16 pair
    for (int k0 = 2 * tid; k0 < p.Kp; k0 += 2 * kOzPrepThreads) {
        unsigned dig[4][kOzPlanes];          // per column, per plane: bits of the pair
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int t = 0; t < kOzPlanes; ++t) dig[j][t] = 0u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = k0 + h;
            if (k >= p.nl || !key_bit(key, p.row0 + k)) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                // active: z = -row
                long long x = p.df ? -(fixed62f(Zh[4 * k + j], e[j]) + fixed62f(Zl[4 * k + j], e[j]))
                                   : fixed62(-Z[4 * k + j], e[j]);
#pragma unroll
                for (int t = 0; t < kOzPlanes; ++t) {
                    const int sh = 56 - 6 * t;
                    const long long d = (x + (1ll << (sh - 1))) >> sh;   // nearest digit
                    x -= d << sh;
                    dig[j][t] |= bf16_of_int((int)d) << (16 * h);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int t = 0; t < kOzPlanes; ++t) {
                const int64_t row = (int64_t)t * p.ncols + 4 * i + j;
                *reinterpret_cast<unsigned *>(p.B + row * p.Kp + k0) = dig[j][t];
            }
    }
}

// ------------------------------------------------------------------------------------------
// rank-1 neighbour compose (Cor. 1 across one flipped neuron, Alg. 1 step 10)

struct R1Init {
    const unsigned long long *keys;
    int kw;
    const int32_t *list;              // items -> cell ids
    const int32_t *parent, *entry;
    const float *prev_rows;           // the parents' level: cell c at (c - prev0) rstride
    int64_t prev0;
    float *rows;                      // this level: cell c at (c - cell0) rstride
    int64_t cell0, rstride;           // floats per cell: 8 (N + 1)
    int L, N;
    int row0[kMaxLayers + 2];         // row0[L + 1] = N
    const double *w_out;
    int *it_l, *it_k;
    float *it_a;                      // per item: a~ as FP32 pairs, [hi x 4 | lo x 4]
};

// (h, l) += d, re-split into an FP32 pair (the rows' 48-bit representation)
__device__ __forceinline__ void pair_add(float &h, float &l, double d)
{
    const double t = (double)h + (double)l + d;
    h = (float)t;
    l = (float)(t - (double)h);
}

// One block per child: the parent's rows of layers 1..l and a_F (the rows of the later layers
// are written by the prep of each layer, from the parent's), row k's sign flipped (s_k flips,
// Z_k does not), and a~ = delta Z_l[k] = the parent's signed row k (its sign (1 - 2 s_k) is
// delta); for a flip in the last layer a_F += w_out[k] a~ and nothing else changes.
__global__ void __launch_bounds__(128) oz_r1_init_kernel(R1Init a)
{
    const int64_t i = blockIdx.x;
    const int64_t c = a.list[i];
    const int64_t p = a.parent[c];
    const int e = a.entry[c];
    int l = a.L;
    for (int ll = 1; ll <= a.L; ++ll)
        if (e < a.row0[ll + 1]) { l = ll; break; }
    const float4 *src = reinterpret_cast<const float4 *>(a.prev_rows + (p - a.prev0) * a.rstride);
    float4 *dst = reinterpret_cast<float4 *>(a.rows + (c - a.cell0) * a.rstride);
    const int lo0 = a.N + 1;                         // the lo block follows the N + 1 hi words
    const int nc = a.row0[l + 1];                    // rows of layers 1..l
#pragma unroll 4
    for (int q = threadIdx.x; q < nc; q += blockDim.x) {
        dst[q] = src[q];
        dst[lo0 + q] = src[lo0 + q];
    }
    __syncthreads();                                 // row e is rewritten below
    if (threadIdx.x != 0) return;
    const float4 h = src[e], lo = src[lo0 + e];
    dst[e] = make_float4(-h.x, -h.y, -h.z, -h.w);
    dst[lo0 + e] = make_float4(-lo.x, -lo.y, -lo.z, -lo.w);
    a.it_l[i] = l;
    a.it_k[i] = e - a.row0[l];
    float *at = a.it_a + 8 * i;
    at[0] = h.x; at[1] = h.y; at[2] = h.z; at[3] = h.w;
    at[4] = lo.x; at[5] = lo.y; at[6] = lo.z; at[7] = lo.w;
    float4 fh = src[a.N], fl = src[lo0 + a.N];
    if (l == a.L) {
        const double w = a.w_out[e - a.row0[l]];
        pair_add(fh.x, fl.x, w * ((double)h.x + (double)lo.x));
        pair_add(fh.y, fl.y, w * ((double)h.y + (double)lo.y));
        pair_add(fh.z, fl.z, w * ((double)h.z + (double)lo.z));
        pair_add(fh.w, fl.w, w * ((double)h.w + (double)lo.w));
    }
    dst[a.N] = fh;
    dst[lo0 + a.N] = fl;
}

struct R1Prep {
    const unsigned long long *keys;
    int kw;
    const int32_t *list;
    const int32_t *parent;
    const float *prev_rows;           // the parents' level: cell c at (c - prev0) rstride
    int64_t prev0;
    float *rows;
    int64_t cell0, rstride;
    int j, L, N, nj, row0j;
    const double *ATj;                // W_j transposed (n_{j-1} x n_j)
    const int *eA;                    // row exponents of W_j
    long long *P, *Q;                 // the products of layer j (items with flip layer <= j - 2), zeroed
    int zero;                         // once read when zero is set (a split-K product)
    int Mp;
    const int *eBin;                  // column exponents of layer j's operand
    int *eBout;                       // column exponents of layer j + 1's operand
    __nv_bfloat16 *B;                 // digit planes of layer j + 1's operand, column = item
    int64_t ncols;
    int Kp;                           // round_up(n_j, 64)
    const double *w_out;
    const int *it_l, *it_k;
    const float *it_a;                // per item: a~ as FP32 pairs, [hi x 4 | lo x 4]
};

// One block per child whose rows of layer j change (flip layer l <= j - 1): v_j (W_j's column k
// when l = j - 1, else the exact product of layer j) as an FP32 pair, the child's rows
// c_j = the parent's + (1 - 2 s_j) v_j a~ in double-float arithmetic (the FP32 pipes: the
// product of the pairs by FMA, TwoSum into the row), and the next operand diag(s_j) v_j as 8
// digit planes (or, at the last layer, a_F += (w_out . diag(s_L) v_L) a~).
__global__ void __launch_bounds__(kOzPrepThreads) oz_r1_prep_kernel(R1Prep a)
{
    constexpr int kW = kOzPrepThreads / 32;
    extern __shared__ float r1v[];                   // diag(s_j) v_j: hi words [0, n_j), lo words [n_j, 2 n_j)
    __shared__ unsigned red[kW];
    __shared__ double fred[kW];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t i = blockIdx.x;
    const int64_t c = a.list[i];
    const unsigned long long *key = a.keys + c * a.kw;
    const float4 *src = reinterpret_cast<const float4 *>(a.prev_rows + (a.parent[c] - a.prev0) * a.rstride);
    float4 *dst = reinterpret_cast<float4 *>(a.rows + (c - a.cell0) * a.rstride);
    const int lo0 = a.N + 1;
    const int l = a.it_l[i];
    float ah[4], al[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        ah[q] = a.it_a[8 * i + q];
        al[q] = a.it_a[8 * i + 4 + q];
    }
    unsigned mx = 0u;
    double fs = 0.0;
    // two rows per thread and pass (n_j = 256 is one pass of 128 threads), every load of both
    // issued before any arithmetic: the kernel is bound by memory latency
    for (int m0 = tid; m0 < a.nj; m0 += 2 * kOzPrepThreads) {
        float4 h4[2], l4[2];
        long long acc[2] = {0, 0};
        double w[2] = {0.0, 0.0};
        int ex[2] = {0, 0};
        bool ok[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int m = m0 + u * kOzPrepThreads;
            ok[u] = m < a.nj;
            if (!ok[u]) continue;
            const int r = a.row0j + m;
            h4[u] = src[r];
            l4[u] = src[lo0 + r];
            if (l == a.j - 1) {
                w[u] = a.ATj[(int64_t)a.it_k[i] * a.nj + m];
            } else {
                const int64_t o = i * a.Mp + m;
                acc[u] = a.P[o] + ((a.Q[o] + 32) >> 6);
                ex[u] = a.eA[m];
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (!ok[u]) continue;
            const int m = m0 + u * kOzPrepThreads;
            float xh, xl;
            if (l == a.j - 1) {
                xh = (float)w[u];
                xl = (float)(w[u] - (double)xh);
            } else {
                if (a.zero) {                         // consumed: zero for the next product's split-K sums
                    const int64_t o = i * a.Mp + m;
                    a.P[o] = 0;
                    a.Q[o] = 0;
                }
                const int e = ex[u] + a.eBin[i] - 48;
                long long hi_int, lo_int;
                xh = i64_to_f32(acc[u], e, &hi_int);
                xl = i64_to_f32(acc[u] - hi_int, e, &lo_int);
            }
            const int r = a.row0j + m;
            const bool act = key_bit(key, r);
            const float sg = act ? -1.0f : 1.0f;     // (1 - 2 s) v
            float h[4] = {h4[u].x, h4[u].y, h4[u].z, h4[u].w}, lo[4] = {l4[u].x, l4[u].y, l4[u].z, l4[u].w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                // (xh + xl)(ah + al) as pp + pe: the exact product of the hi words by FMA, the two
                // cross terms into its error (xl al, below 2^-48 of the product, is dropped)
                const float pp = xh * ah[q];
                float pe = fmaf(xh, ah[q], -pp);
                pe = fmaf(xh, al[q], pe);
                pe = fmaf(xl, ah[q], pe);
                df_add(h[q], lo[q], sg * pp, sg * pe);
                df_norm(h[q], lo[q]);
            }
            dst[r] = make_float4(h[0], h[1], h[2], h[3]);
            dst[lo0 + r] = make_float4(lo[0], lo[1], lo[2], lo[3]);
            r1v[m] = act ? xh : 0.0f;
            r1v[a.nj + m] = act ? xl : 0.0f;
            if (act) {
                const unsigned b = __float_as_uint(xh) & 0x7FFFFFFFu;
                mx = b > mx ? b : mx;
                if (a.j == a.L) fs = fma(a.w_out[m], (double)xh + (double)xl, fs);
            }
        }
    }
    if (a.j == a.L) {
        for (int o = 16; o > 0; o >>= 1) fs += __shfl_xor_sync(0xffffffffu, fs, o);
        if (lane == 0) fred[wid] = fs;
        __syncthreads();
        if (tid == 0) {
            double f = 0.0;
            for (int w = 0; w < kW; ++w) f += fred[w];
            float4 fh = dst[a.N], fl = dst[lo0 + a.N];
            pair_add(fh.x, fl.x, f * ((double)ah[0] + (double)al[0]));
            pair_add(fh.y, fl.y, f * ((double)ah[1] + (double)al[1]));
            pair_add(fh.z, fl.z, f * ((double)ah[2] + (double)al[2]));
            pair_add(fh.w, fl.w, f * ((double)ah[3] + (double)al[3]));
            dst[a.N] = fh;
            dst[lo0 + a.N] = fl;
        }
        return;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned v = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = v > mx ? v : mx;
    }
    if (lane == 0) red[wid] = mx;
    __syncthreads();
    unsigned m2 = 0u;
    for (int w = 0; w < kW; ++w) m2 = red[w] > m2 ? red[w] : m2;
    // |hi + lo| <= |hi| (1 + 2^-24): one binade of headroom above the largest |hi|
    const int be = (int)(m2 >> 23);
    const int e = m2 == 0u ? 0 : (be == 0 ? -126 : be - 127 + 1);
    if (tid == 0) a.eBout[i] = e;
    for (int k0 = 2 * tid; k0 < a.Kp; k0 += 2 * kOzPrepThreads) {
        unsigned dig[kOzPlanes];
#pragma unroll
        for (int t = 0; t < kOzPlanes; ++t) dig[t] = 0u;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int k = k0 + hh;
            if (k >= a.nj) continue;
            long long x = fixed62f(r1v[k], e) + fixed62f(r1v[a.nj + k], e);
#pragma unroll
            for (int t = 0; t < kOzPlanes; ++t) {
                const int sh = 56 - 6 * t;
                const long long d = (x + (1ll << (sh - 1))) >> sh;   // nearest digit
                x -= d << sh;
                dig[t] |= bf16_of_int((int)d) << (16 * hh);
            }
        }
#pragma unroll
        for (int t = 0; t < kOzPlanes; ++t)
            *reinterpret_cast<unsigned *>(a.B + ((int64_t)t * a.ncols + i) * a.Kp + k0) = dig[t];
    }
}

// the cells [c_begin, n) of the next level: rank-1 from the parent when it lies in [p0, p1)
// and its chain of rank-1 composes is below max_chain - 1, else a full compose
__global__ void oz_r1_classify_kernel(Arena ar, int64_t p0, int64_t p1, int64_t c_begin, int max_chain, int L,
                                      R1Rows rr, unsigned long long *counts)
{
    const unsigned long long nc = __ldcg(ar.counters + kNCells);
    const int64_t n = (int64_t)nc < ar.cap ? (int64_t)nc : ar.cap;
    for (int64_t c = c_begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = ar.parent[c];
        const int e = ar.entry_plane[c];
        int cls = -1;
        if (p >= p0 && p < p1 && e >= 0) {
            const int ch = ar.chain[p];
            if (ch + 1 < max_chain) {
                cls = L;
                for (int ll = 1; ll <= L; ++ll)
                    if (e < rr.row0[ll + 1]) { cls = ll; break; }
                ar.chain[c] = ch + 1;
            }
        }
        if (cls < 0) ar.chain[c] = 0;
        ar.cls[c] = cls;
        atomicAdd(counts + (cls < 0 ? 0 : cls), 1ull);
    }
}

__global__ void oz_r1_scatter_kernel(Arena ar, int64_t c0, int64_t c1, int32_t *full, int32_t *r1, int *offs)
{
    for (int64_t c = c0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < c1; c += (int64_t)gridDim.x * blockDim.x) {
        const int cls = ar.cls[c];
        if (cls < 0) full[atomicAdd(offs + kMaxLayers + 1, 1)] = (int32_t)c;
        else r1[offs[cls] + atomicAdd(offs + kMaxLayers + 1 + cls, 1)] = (int32_t)c;
    }
}

// ------------------------------------------------------------------------------------------
// the layer product on the tensor cores

struct OzGemm {
    int64_t ncols_used;               // columns [0, ncols_used) are written (every one has a consumer)
    long long *P;                     // exact products of diagonals 0..6, column c at P + c Mp (rows 0..Mp-1)
    long long *Q;                     // the raw sum of diagonal 7, same layout (rounded once, by the prep)
    int Mp;                           // row stride between digit planes of W_l, and of P
    int64_t n;                        // cells in the batch
    int KC;                           // K chunks (Kp / 64) of the whole product
    int split;                        // K chunks split over gridDim.z CTAs: partial sums added atomically
    int64_t ncols;                    // column stride between digit planes of B
    int *err;
};

template <int NC, int AST>
struct OzShape {
    static constexpr int kNCol = 4 * NC;                       // UMMA N
    static constexpr int kATile = kOzM * 128;                  // bytes of one A stage
    static constexpr int kBPlane = kNCol * 128;                // bytes of one B digit-plane tile
    static constexpr int kBStage = kOzPlanes * kBPlane;
    static constexpr int kTmemCols = kOzPlanes * kNCol;        // 8 diagonals
    static constexpr int kBars = 2 * AST + 2 * 2 + 2;
    static constexpr int kSmem = AST * kATile + 2 * kBStage + kBars * 8 + 16 + 1024;
    static_assert(kTmemCols == 256 || kTmemCols == 512, "TMEM allocation must be a power of two");
    static_assert(kBPlane % 1024 == 0, "B plane tiles must stay 1024-byte aligned");
};

template <int NC, int AST>
__global__ void __launch_bounds__(192, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzGemm g)
{
    using S = OzShape<NC, AST>;
    extern __shared__ unsigned char oz_smem_raw[];
    const uint32_t raw = smem_u32(oz_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = oz_smem_raw + (base - raw);
    const uint32_t sA = base, sB = base + AST * S::kATile;
    const uint32_t bars = sB + 2 * S::kBStage;
    auto afull = [&](int q) { return bars + 8 * q; };
    auto aempty = [&](int q) { return bars + 8 * (AST + q); };
    auto bfull = [&](int q) { return bars + 8 * (2 * AST + q); };
    auto bempty = [&](int q) { return bars + 8 * (2 * AST + 2 + q); };
    const uint32_t accfull = bars + 8 * (2 * AST + 4), drain = bars + 8 * (2 * AST + 5);
    unsigned char *tail = gbase + (bars - base) + 8 * S::kBars;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tail);
    volatile int *abort = reinterpret_cast<volatile int *>(tail + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kOzM;
    const int64_t col0 = (int64_t)blockIdx.y * S::kNCol;
    // K chunks [kc0, kc0 + nkc) of this CTA (split-K over gridDim.z)
    const int kc0 = (int)((int64_t)g.KC * blockIdx.z / gridDim.z);
    const int nkc = (int)((int64_t)g.KC * (blockIdx.z + 1) / gridDim.z) - kc0;

    if (threadIdx.x == 0) {
        for (int q = 0; q < AST; ++q) { mbar_init(afull(q), 1); mbar_init(aempty(q), 1); }
        for (int q = 0; q < 2; ++q) { mbar_init(bfull(q), 1); mbar_init(bempty(q), 1); }
        mbar_init(accfull, 1);
        mbar_init(drain, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(S::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- producer: per K chunk the 8 digit planes of the stacked operand, then the 8
        //      digit planes of W_l one at a time
        if (lane == 0) {
            int armedA[AST], armedB[2];
            for (int q = 0; q < AST; ++q) armedA[q] = 0;
            armedB[0] = armedB[1] = 0;
            int ai = 0;
            bool ok = true;
            for (int it = 0; it < nkc && ok; ++it) {
                const int kc = kc0 + it, bs = it & 1;
                if (it >= 2 && !mbar_wait(bempty(bs), ((it >> 1) - 1) & 1, abort, g.err)) { ok = false; break; }
                mbar_expect_tx(bfull(bs), S::kBStage);
                ++armedB[bs];
                for (int t = 0; t < kOzPlanes; ++t)
                    tma_load_2d(sB + bs * S::kBStage + t * S::kBPlane, &tmB, kc * kOzBK,
                                (int)((int64_t)t * g.ncols + col0), bfull(bs));
                for (int s = 0; s < kOzPlanes; ++s, ++ai) {
                    const int q = ai % AST;
                    if (ai >= AST && !mbar_wait(aempty(q), ((ai / AST) - 1) & 1, abort, g.err)) { ok = false; break; }
                    mbar_expect_tx(afull(q), S::kATile);
                    ++armedA[q];
                    tma_load_2d(sA + q * S::kATile, &tmA, kc * kOzBK, s * g.Mp + m0, afull(q));
                }
            }
            if (!ok) {
                // let every copy already issued land before the CTA's shared memory goes away
                for (int q = 0; q < AST; ++q)
                    if (armedA[q]) mbar_drain(afull(q), (armedA[q] - 1) & 1, kOzDrainNs);
                for (int q = 0; q < 2; ++q)
                    if (armedB[q]) mbar_drain(bfull(q), (armedB[q] - 1) & 1, kOzDrainNs);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer: plane s of W_l times planes t = 0..7-s of the operand, into the
        //      accumulator of diagonal s + t
        if (lane == 0) {
            int ai = 0;
            bool ok = true;
            for (int it = 0; it < nkc && ok; ++it) {
                const int bs = it & 1;
                if (!mbar_wait(bfull(bs), (it >> 1) & 1, abort, g.err)) { ok = false; break; }
                for (int s = 0; s < kOzPlanes; ++s, ++ai) {
                    const int q = ai % AST;
                    if (!mbar_wait(afull(q), (ai / AST) & 1, abort, g.err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a0 = sA + q * S::kATile;
                    const uint64_t adesc = sw128_desc(a0), bdesc = sw128_desc(sB + bs * S::kBStage);
                    const uint32_t acc0 = (it | s) != 0 ? 1u : 0u;
                    switch (kOzPlanes - s) {                  // operand planes t = 0 .. 7 - s
                    case 8: issue_plane<8, S::kNCol, S::kBPlane>(tmem, s, adesc, bdesc, acc0); break;
                    case 7: issue_plane<7, S::kNCol, S::kBPlane>(tmem, s, adesc, bdesc, acc0); break;
                    case 6: issue_plane<6, S::kNCol, S::kBPlane>(tmem, s, adesc, bdesc, acc0); break;
                    case 5: issue_plane<5, S::kNCol, S::kBPlane>(tmem, s, adesc, bdesc, acc0); break;
                    case 4: issue_plane<4, S::kNCol, S::kBPlane>(tmem, s, adesc, bdesc, acc0); break;
                    case 3: issue_plane<3, S::kNCol, S::kBPlane>(tmem, s, adesc, bdesc, acc0); break;
                    case 2: issue_plane<2, S::kNCol, S::kBPlane>(tmem, s, adesc, bdesc, acc0); break;
                    default: issue_plane<1, S::kNCol, S::kBPlane>(tmem, s, adesc, bdesc, acc0); break;
                    }
                    umma_commit(aempty(q));          // the A stage is free once these products finish
                }
                if (ok) umma_commit(bempty(bs));
            }
            if (ok) {
                umma_commit(accfull);
            } else {
                umma_commit(drain);                  // every product issued so far has finished
                mbar_drain(drain, 0, kOzDrainNs);
            }
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, one row of W_l per thread,
        //      and writes the exact product of each column as a 64-bit integer at scale 2^-48
        //      (the prep kernel applies the exponents, C_l and the sign)
        const int quarter = warp & 3;
        const int grow = m0 + quarter * 32 + lane;
        if (mbar_wait(accfull, 0, abort, g.err)) {
            tc_fence_after();
            const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
            for (int c2 = 0; c2 < NC; c2 += 2) {
                // 8 columns (two cells) of all 8 diagonals, one wait for the lot
                uint32_t v[kOzPlanes][8];
#pragma unroll
                for (int dg = 0; dg < kOzPlanes; ++dg) tmem_ld8_nowait(trow + (uint32_t)(dg * S::kNCol + 4 * c2), v[dg]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    long long a = (long long)__float2int_rn(__uint_as_float(v[0][j]));
#pragma unroll
                    for (int dg = 1; dg < kOzPlanes - 1; ++dg) a = (a << 6) + (long long)__float2int_rn(__uint_as_float(v[dg][j]));
                    const long long a7 = (long long)__float2int_rn(__uint_as_float(v[kOzPlanes - 1][j]));
                    const int64_t col = col0 + 4 * c2 + j;
                    if (col < g.ncols_used) {
                        long long *dst = g.P + col * g.Mp + grow, *dq = g.Q + col * g.Mp + grow;
                        if (g.split) {
                            atomicAdd(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)a);
                            atomicAdd(reinterpret_cast<unsigned long long *>(dq), (unsigned long long)a7);
                        } else {
                            *dst = a;
                            *dq = a7;
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::kTmemCols) : "memory");
    }
}

// ------------------------------------------------------------------------------------------
// the wide tile: 32 cells (UMMA N = 128), the diagonals in two passes
//
// A stream of M = 128 products from one CTA costs at least about 71 clock cycles per
// instruction for any N <= 128 (measured on this part), so N = 64 tiles reach at most 45 % of
// the tensor peak and N = 128 tiles 90 %.  All 8 diagonal accumulators at N = 128 would need
// 1024 TMEM columns, so this tile keeps 4 at a time: pass 1 accumulates diagonals 0..3, the
// epilogue drains them (exact 64-bit integers), pass 2 accumulates diagonals 4..7 into the same
// columns.  Pass 2 runs as two sweeps over K, operand planes 0..3 then 4..7, so that a B stage
// holds 4 planes (64 KB) and two stages fit beside six A stages.

template <int SW> struct OzSweep;     // diagonal base, operand planes [tlo, thi], W planes [slo, shi]
template <> struct OzSweep<0> { static constexpr int base = 0, tlo = 0, thi = 3, slo = 0, shi = 3; };
template <> struct OzSweep<1> { static constexpr int base = 4, tlo = 0, thi = 3, slo = 1, shi = 7; };
template <> struct OzSweep<2> { static constexpr int base = 4, tlo = 4, thi = 7, slo = 0, shi = 3; };

constexpr int oz_imax(int a, int b) { return a > b ? a : b; }
constexpr int oz_imin(int a, int b) { return a < b ? a : b; }

// The products of W plane SS with the sweep's operand planes whose diagonal lies in
// [base, base + 3], for the 4 K steps of a chunk, A kept in the collector per K step.  init:
// bit j set once accumulator j holds a value (its first product overwrites).
template <int SW, int SS, int NCOL, int BPLANE>
__device__ __forceinline__ void oz_issue_wide(uint32_t tmem, uint64_t adesc, uint64_t bdesc, unsigned &init)
{
    using W = OzSweep<SW>;
    constexpr int t0 = oz_imax(W::tlo, W::base - SS), t1 = oz_imin(W::thi, W::base + 3 - SS);
    if constexpr (t1 >= t0) {
        constexpr int cnt = t1 - t0 + 1;
        constexpr uint32_t idesc = umma_idesc_bf16(128, NCOL);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = adesc + (uint64_t)(2 * kk);
#pragma unroll
            for (int t = t0; t <= t1; ++t) {
                const int slot = SS + t - W::base;
                const uint64_t bd = bdesc + (uint64_t)(((t - W::tlo) * BPLANE + 32 * kk) >> 4);
                const uint32_t d = tmem + (uint32_t)(slot * NCOL);
                const uint32_t acc = (init >> slot) & 1u;
                init |= 1u << slot;
                if constexpr (cnt == 1) umma_bf16(d, ad, bd, idesc, acc);
                else if (t == t0) umma_bf16_collect<1>(d, ad, bd, idesc, acc);
                else if (t < t1) umma_bf16_collect<2>(d, ad, bd, idesc, acc);
                else umma_bf16_collect<3>(d, ad, bd, idesc, acc);
            }
        }
    }
}

template <int SW, int NCOL, int BPLANE>
__device__ __forceinline__ void oz_issue_wide_s(int s, uint32_t tmem, uint64_t adesc, uint64_t bdesc, unsigned &init)
{
    switch (s) {
    case 0: oz_issue_wide<SW, 0, NCOL, BPLANE>(tmem, adesc, bdesc, init); break;
    case 1: oz_issue_wide<SW, 1, NCOL, BPLANE>(tmem, adesc, bdesc, init); break;
    case 2: oz_issue_wide<SW, 2, NCOL, BPLANE>(tmem, adesc, bdesc, init); break;
    case 3: oz_issue_wide<SW, 3, NCOL, BPLANE>(tmem, adesc, bdesc, init); break;
    case 4: oz_issue_wide<SW, 4, NCOL, BPLANE>(tmem, adesc, bdesc, init); break;
    case 5: oz_issue_wide<SW, 5, NCOL, BPLANE>(tmem, adesc, bdesc, init); break;
    case 6: oz_issue_wide<SW, 6, NCOL, BPLANE>(tmem, adesc, bdesc, init); break;
    default: oz_issue_wide<SW, 7, NCOL, BPLANE>(tmem, adesc, bdesc, init); break;
    }
}

__host__ __device__ constexpr int oz_sweep_slo(int sw) { return sw == 1 ? 1 : 0; }
__host__ __device__ constexpr int oz_sweep_shi(int sw) { return sw == 1 ? 7 : 3; }
__host__ __device__ constexpr int oz_sweep_tlo(int sw) { return sw == 2 ? 4 : 0; }

template <int AST>
struct OzWideShape {
    static constexpr int kNCol = 128;                          // 32 cells
    static constexpr int kATile = kOzM * 128;
    static constexpr int kBPlane = kNCol * 128;                // 16 KB
    static constexpr int kBStage = 4 * kBPlane;                // 4 operand planes
    static constexpr int kTmemCols = 4 * kNCol;                // 4 diagonals at a time
    static constexpr int kBars = 2 * AST + 2 * 2 + 3;
    static constexpr int kSmem = AST * kATile + 2 * kBStage + kBars * 8 + 16 + 1024;
    static_assert(kSmem <= 232448, "shared memory");
};

template <int AST>
__global__ void __launch_bounds__(320, 1)
    oz_gemm_wide_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzGemm g)
{
    using S = OzWideShape<AST>;
    extern __shared__ unsigned char oz_smem_raw[];
    const uint32_t raw = smem_u32(oz_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = oz_smem_raw + (base - raw);
    const uint32_t sA = base, sB = base + AST * S::kATile;
    const uint32_t bars = sB + 2 * S::kBStage;
    auto afull = [&](int q) { return bars + 8 * q; };
    auto aempty = [&](int q) { return bars + 8 * (AST + q); };
    auto bfull = [&](int q) { return bars + 8 * (2 * AST + q); };
    auto bempty = [&](int q) { return bars + 8 * (2 * AST + 2 + q); };
    const uint32_t accfull = bars + 8 * (2 * AST + 4), drain = bars + 8 * (2 * AST + 5),
                   tmem_empty = bars + 8 * (2 * AST + 6);
    unsigned char *tail = gbase + (bars - base) + 8 * S::kBars;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tail);
    volatile int *abort = reinterpret_cast<volatile int *>(tail + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kOzM;
    const int64_t col0 = (int64_t)blockIdx.y * S::kNCol;
    const int kc0 = (int)((int64_t)g.KC * blockIdx.z / gridDim.z);
    const int nkc = (int)((int64_t)g.KC * (blockIdx.z + 1) / gridDim.z) - kc0;

    if (threadIdx.x == 0) {
        for (int q = 0; q < AST; ++q) { mbar_init(afull(q), 1); mbar_init(aempty(q), 1); }
        for (int q = 0; q < 2; ++q) { mbar_init(bfull(q), 1); mbar_init(bempty(q), 1); }
        mbar_init(accfull, 1);
        mbar_init(drain, 1);
        mbar_init(tmem_empty, 8);                 // one arrival per epilogue warp
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(S::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- producer: three sweeps over this CTA's K chunks; per chunk the sweep's 4 operand
        //      planes, then its W planes one at a time
        if (lane == 0) {
            int armedA[AST], armedB[2];
            for (int q = 0; q < AST; ++q) armedA[q] = 0;
            armedB[0] = armedB[1] = 0;
            int ai = 0, bi = 0;
            bool ok = true;
            for (int sw = 0; sw < 3 && ok; ++sw) {
                for (int it = 0; it < nkc && ok; ++it, ++bi) {
                    const int kc = kc0 + it, bs = bi & 1;
                    if (bi >= 2 && !mbar_wait(bempty(bs), ((bi >> 1) - 1) & 1, abort, g.err)) { ok = false; break; }
                    mbar_expect_tx(bfull(bs), S::kBStage);
                    ++armedB[bs];
                    for (int t = 0; t < 4; ++t)
                        tma_load_2d(sB + bs * S::kBStage + t * S::kBPlane, &tmB, kc * kOzBK,
                                    (int)((int64_t)(oz_sweep_tlo(sw) + t) * g.ncols + col0), bfull(bs));
                    for (int sp = oz_sweep_slo(sw); sp <= oz_sweep_shi(sw); ++sp, ++ai) {
                        const int q = ai % AST;
                        if (ai >= AST && !mbar_wait(aempty(q), ((ai / AST) - 1) & 1, abort, g.err)) { ok = false; break; }
                        mbar_expect_tx(afull(q), S::kATile);
                        ++armedA[q];
                        tma_load_2d(sA + q * S::kATile, &tmA, kc * kOzBK, sp * g.Mp + m0, afull(q));
                    }
                }
            }
            if (!ok) {
                for (int q = 0; q < AST; ++q)
                    if (armedA[q]) mbar_drain(afull(q), (armedA[q] - 1) & 1, kOzDrainNs);
                for (int q = 0; q < 2; ++q)
                    if (armedB[q]) mbar_drain(bfull(q), (armedB[q] - 1) & 1, kOzDrainNs);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            int ai = 0, bi = 0;
            bool ok = true;
            unsigned init = 0u;
            for (int sw = 0; sw < 3 && ok; ++sw) {
                if (sw == 1) {
                    // pass 2 reuses the accumulators: wait until the epilogue has read pass 1
                    if (!mbar_wait(tmem_empty, 0, abort, g.err)) { ok = false; break; }
                    tc_fence_after();
                    init = 0u;
                }
                for (int it = 0; it < nkc && ok; ++it, ++bi) {
                    const int bs = bi & 1;
                    if (!mbar_wait(bfull(bs), (bi >> 1) & 1, abort, g.err)) { ok = false; break; }
                    for (int sp = oz_sweep_slo(sw); sp <= oz_sweep_shi(sw); ++sp, ++ai) {
                        const int q = ai % AST;
                        if (!mbar_wait(afull(q), (ai / AST) & 1, abort, g.err)) { ok = false; break; }
                        tc_fence_after();
                        const uint64_t ad = sw128_desc(sA + q * S::kATile), bd = sw128_desc(sB + bs * S::kBStage);
                        if (sw == 0) oz_issue_wide_s<0, S::kNCol, S::kBPlane>(sp, tmem, ad, bd, init);
                        else if (sw == 1) oz_issue_wide_s<1, S::kNCol, S::kBPlane>(sp, tmem, ad, bd, init);
                        else oz_issue_wide_s<2, S::kNCol, S::kBPlane>(sp, tmem, ad, bd, init);
                        umma_commit(aempty(q));
                    }
                    if (ok) umma_commit(bempty(bs));
                }
                if (ok && sw != 1) umma_commit(accfull);     // after pass 1 (sweep 0) and pass 2 (sweep 2)
            }
            if (!ok) {
                umma_commit(drain);
                mbar_drain(drain, 0, kOzDrainNs);
            }
        }
    } else {
        // ---- epilogue (warps 2..9, two per TMEM lane quarter, each half of the columns): twice,
        //      once per pass; exact 64-bit products
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int grow = m0 + quarter * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
        for (int pass = 0; pass < 2; ++pass) {
            if (!mbar_wait(accfull, pass, abort, g.err)) break;
            tc_fence_after();
#pragma unroll 1
            for (int c8 = half * (S::kNCol / 2); c8 < (half + 1) * (S::kNCol / 2); c8 += 8) {
                uint32_t v[4][8];
#pragma unroll
                for (int dg = 0; dg < 4; ++dg) tmem_ld8_nowait(trow + (uint32_t)(dg * S::kNCol + c8), v[dg]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    long long a;
                    if (pass == 0) {         // D0 2^36 + D1 2^30 + D2 2^24 + D3 2^18
                        a = (long long)__float2int_rn(__uint_as_float(v[0][j]));
#pragma unroll
                        for (int dg = 1; dg < 4; ++dg) a = (a << 6) + (long long)__float2int_rn(__uint_as_float(v[dg][j]));
                        a <<= 18;
                    } else {                 // D4 2^18 + D5 2^12 + D6 2^6 + D7, at scale 2^-54, to Q
                        a = (long long)__float2int_rn(__uint_as_float(v[0][j]));
#pragma unroll
                        for (int dg = 1; dg < 4; ++dg) a = (a << 6) + (long long)__float2int_rn(__uint_as_float(v[dg][j]));
                    }
                    // pass 1 to P, pass 2 to Q: the prep's P + round(Q / 64) adds them exactly,
                    // so neither pass reads the other's result back
                    const int64_t col = col0 + c8 + j;
                    if (col < g.ncols_used) {
                        long long *dst = (pass ? g.Q : g.P) + col * g.Mp + grow;
                        if (g.split) atomicAdd(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)a);
                        else *dst = a;
                    }
                }
            }
            if (pass == 0) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tmem_empty) : "memory");
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::kTmemCols) : "memory");
    }
}

// ------------------------------------------------------------------------------------------
// host side

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encode()
{
    if (g_encode) return cudaSuccess;
    cudaDriverEntryPointQueryResult q{};
    void *fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return cudaSuccess;
}

// 2-D BF16 tensor of `rows` rows of Kp elements, boxes of 64 x box_rows with the 128-byte swizzle
cudaError_t encode_map(CUtensorMap *m, const void *ptr, int64_t Kp, int64_t rows, int box_rows)
{
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kOzBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int NC, int AST>
cudaError_t launch_gemm(const CUtensorMap &tmA, const CUtensorMap &tmB, const OzGemm &g, int Mp, int64_t ncols_used,
                        int split, cudaStream_t st)
{
    using S = OzShape<NC, AST>;
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel<NC, AST>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kSmem);
    if (e != cudaSuccess) return e;
    const dim3 grid(Mp / kOzM, (unsigned)((ncols_used + S::kNCol - 1) / S::kNCol), (unsigned)split);
    oz_gemm_kernel<NC, AST><<<grid, 192, S::kSmem, st>>>(tmA, tmB, g);
    return cudaGetLastError();
}

template <int AST>
cudaError_t launch_gemm_wide(const CUtensorMap &tmA, const CUtensorMap &tmB, const OzGemm &g, int Mp,
                             int64_t ncols_used, int split, cudaStream_t st)
{
    using S = OzWideShape<AST>;
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_wide_kernel<AST>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kSmem);
    if (e != cudaSuccess) return e;
    const dim3 grid(Mp / kOzM, (unsigned)((ncols_used + S::kNCol - 1) / S::kNCol), (unsigned)split);
    oz_gemm_wide_kernel<AST><<<grid, 320, S::kSmem, st>>>(tmA, tmB, g);
    return cudaGetLastError();
}

}  // namespace

int oz_kp(int width) { return (width + kOzBK - 1) / kOzBK * kOzBK; }
int oz_mp(int width) { return (width + kOzM - 1) / kOzM * kOzM; }

const int *oz_tile_cells(int *n)
{
    static const int cells[] = {0, 32, 16, 8};     // 0: automatic per batch
    *n = 4;
    return cells;
}

// Digit planes of the hidden part of W_l (n rows, np columns, row stride fan): plane s row m at
// (s Mp + m) Kp, zero padded; the row exponents eA (n values).  Host arithmetic, exact.
void oz_slice_weights(const double *W, int n, int np, int fan, std::vector<uint16_t> &planes, std::vector<int> &eA)
{
    const int Kp = oz_kp(np), Mp = oz_mp(n);
    planes.assign((size_t)kOzPlanes * Mp * Kp, 0);
    eA.assign(n, 0);
    for (int m = 0; m < n; ++m) {
        double mx = 0.0;
        for (int k = 0; k < np; ++k) mx = std::max(mx, std::fabs(W[(size_t)m * fan + k]));
        int e = 0;
        if (mx > 0.0) {
            int ex;
            const double fr = std::frexp(mx, &ex);       // mx = fr 2^ex, fr in [0.5, 1)
            e = fr == 0.5 ? ex - 1 : ex;                 // smallest e with mx <= 2^e
        }
        eA[m] = e;
        for (int k = 0; k < np; ++k) {
            double x = std::ldexp(W[(size_t)m * fan + k], -e);   // |x| <= 1, exact
            for (int s = 0; s < kOzPlanes; ++s) {
                const double t = std::ldexp(x, kOzBeta);
                const double d = std::nearbyint(t);              // |d| <= 64 (s = 0), <= 32 after
                x = t - d;                                       // exact, |x| <= 1/2
                float f = (float)d;
                uint32_t u;
                std::memcpy(&u, &f, 4);
                planes[((size_t)s * Mp + m) * Kp + k] = (uint16_t)(u >> 16);
            }
        }
    }
}

cudaError_t oz_encode_weights(void *map, const void *planes, int n, int np)
{
    return encode_map(reinterpret_cast<CUtensorMap *>(map), planes, oz_kp(np), (int64_t)kOzPlanes * oz_mp(n), kOzM);
}

int64_t oz_scratch_elems(int64_t batch_cells, int max_kp)
{
    return (int64_t)kOzPlanes * 4 * batch_cells * max_kp;
}

// One layer's product on the tensor cores: the digit planes of W_l (net.mapA[l]) times the
// first ncols_used columns of the stacked operand (scr.B, written by the previous prep) into the
// exact products P, Q.  The tile shape: tile_cells, or (0) the 32-cell tile when K has at least 8
// chunks (its two passes' fixed costs amortise) and its tiles, split over up to 4 K ranges, fill
// every SM, else the 16-cell tile, which makes twice as many.  A product too small to fill the
// SMs splits K over more CTAs (exact integer sums) that add into P and Q, which must then be zero:
// *split_out tells the caller's prep to zero what it reads, and a product that writes without
// splitting leaves P and Q dirty (a memset then precedes the next split product).
static cudaError_t oz_layer_product(const OzNet &net, int l, const OzScratch &scr, int64_t ncols_used, int tile_cells,
                                    int sms, cudaStream_t st, int *split_out)
{
    const int64_t ncols = 4 * scr.batch_cells;
    const int Mp = oz_mp(net.width[l]);
    const int Kp = oz_kp(net.width[l - 1]);
    const int64_t nb = (ncols_used + 3) / 4;                  // in units of 4 columns
    const int tc = tile_cells ? tile_cells
                              : (Kp / kOzBK >= 8 && (int64_t)(Mp / kOzM) * ((4 * nb + 127) / 128) * 4 >= sms ? 32 : 16);
    const int per_sm = tc == 8 ? 2 : 1;                       // resident tiles per SM (shared memory)
    CUtensorMap tmB;
    cudaError_t e = encode_map(&tmB, scr.B, Kp, (int64_t)kOzPlanes * ncols, 4 * tc);
    if (e != cudaSuccess) return e;
    OzGemm g{};
    g.P = scr.P;
    g.Q = scr.Q;
    g.Mp = Mp;
    g.n = nb;
    g.KC = Kp / kOzBK;
    g.ncols = ncols;
    g.err = scr.err;
    g.ncols_used = ncols_used;
    const int64_t tiles = (int64_t)(g.Mp / kOzM) * ((4 * nb + 4 * tc - 1) / (4 * tc));
    int split = (int)std::min<int64_t>(std::min<int64_t>(g.KC, 4), std::max<int64_t>(1, (int64_t)sms * per_sm / tiles));
    g.split = split > 1 ? 1 : 0;
    *split_out = g.split;
    if (g.split) {
        if (scr.dirty && *scr.dirty > 0) {
            e = cudaMemsetAsync(scr.P, 0, sizeof(long long) * *scr.dirty, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(scr.Q, 0, sizeof(long long) * *scr.dirty, st);
            if (e != cudaSuccess) return e;
            *scr.dirty = 0;
        }
    } else if (scr.dirty) {
        *scr.dirty = std::max<int64_t>(*scr.dirty, ncols_used * (int64_t)g.Mp);
    }
    const CUtensorMap &tmA = *reinterpret_cast<const CUtensorMap *>(net.mapA[l]);
    // 36 digit-plane products per layer over the padded tiles of the columns in use
    if (scr.issued) *scr.issued += (int64_t)36 * (4 * nb) * Mp * Kp;
    return tc == 8    ? launch_gemm<8, 2>(tmA, tmB, g, g.Mp, 4 * nb, split, st)
           : tc == 32 ? launch_gemm_wide<6>(tmA, tmB, g, g.Mp, 4 * nb, split, st)
                      : launch_gemm<16, 6>(tmA, tmB, g, g.Mp, 4 * nb, split, st);
}

cudaError_t oz_compose(const OzNet &net, const unsigned long long *keys, int kw, int64_t n, void *rows, bool df,
                       const OzScratch &scr, int tile_cells, int sms, cudaStream_t st, const int32_t *list,
                       int64_t cell0)
{
    const int64_t rstride = 4 * (int64_t)(net.N + 1);
    const int64_t ncols = 4 * scr.batch_cells;

    for (int64_t b0 = 0; b0 < n; b0 += scr.batch_cells) {
        const int64_t nb = std::min<int64_t>(scr.batch_cells, n - b0);
        OzPrep p{};
        p.keys = list ? keys : keys + b0 * kw;
        p.list = list ? list + b0 : nullptr;
        p.cell0 = cell0;
        p.kw = kw;
        p.n = nb;
        p.rows = list ? rows : reinterpret_cast<double *>(rows) + b0 * rstride;
        p.rstride = rstride;
        p.df = df ? 1 : 0;
        p.L = net.L;
        p.N = net.N;
        p.w_out = net.w_out;
        p.b_out = net.b_out;
        p.B = scr.B;
        p.P = scr.P;
        p.Q = scr.Q;
        p.ncols = ncols;
        for (int l = 1; l <= net.L; ++l) {
            p.eBin = scr.eB[l & 1];                    // written by the prep of layer l - 1
            p.eBout = scr.eB[(l + 1) & 1];
            p.zero = 0;
            if (l >= 2) {
                cudaError_t e = oz_layer_product(net, l, scr, 4 * nb, tile_cells, sms, st, &p.zero);
                if (e != cudaSuccess) return e;
                p.Mp = oz_mp(net.width[l]);
                p.eA = net.eA[l];
            }
            p.l = l;
            p.nl = net.width[l];
            p.row0 = net.row0[l];
            p.Cl = net.Cl[l];
            p.Clhi = net.Clhi[l];
            p.Cllo = net.Cllo[l];
            p.Kp = oz_kp(net.width[l]);
            oz_prep_kernel<<<(unsigned)nb, kOzPrepThreads, 0, st>>>(p);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}


// row i = cell c = i / per, row k = i % per: the cell's pairs hold its `per` hi words, then its
// `per` lo words
__device__ __forceinline__ int64_t pair_hi(int64_t i, int per) { return (i / per) * 2 * per + i % per; }

__global__ void rows_to_pairs_kernel(const double *rows, float *pairs, int64_t nrows, int per)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x) {
        float h[4], l[4];
        for (int q = 0; q < 4; ++q) {
            const double v = rows[4 * i + q];
            h[q] = (float)v;
            l[q] = (float)(v - (double)h[q]);
        }
        const int64_t o = pair_hi(i, per);
        reinterpret_cast<float4 *>(pairs)[o] = make_float4(h[0], h[1], h[2], h[3]);
        reinterpret_cast<float4 *>(pairs)[o + per] = make_float4(l[0], l[1], l[2], l[3]);
    }
}

__global__ void pairs_to_rows_kernel(const float *pairs, double *rows, int64_t nrows, int per)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = pair_hi(i, per);
        const float4 h = reinterpret_cast<const float4 *>(pairs)[o], l = reinterpret_cast<const float4 *>(pairs)[o + per];
        rows[4 * i] = (double)h.x + (double)l.x;
        rows[4 * i + 1] = (double)h.y + (double)l.y;
        rows[4 * i + 2] = (double)h.z + (double)l.z;
        rows[4 * i + 3] = (double)h.w + (double)l.w;
    }
}

void rows_to_pairs(const double *rows, float *pairs, int64_t n_cells, int rows_per_cell, cudaStream_t st)
{
    const int64_t nrows = n_cells * rows_per_cell;
    rows_to_pairs_kernel<<<(unsigned)std::min<int64_t>((nrows + 255) / 256, 152 * 16), 256, 0, st>>>(rows, pairs, nrows,
                                                                                                    rows_per_cell);
}

void pairs_to_rows(const float *pairs, double *rows, int64_t n_cells, int rows_per_cell, cudaStream_t st)
{
    const int64_t nrows = n_cells * rows_per_cell;
    pairs_to_rows_kernel<<<(unsigned)std::min<int64_t>((nrows + 255) / 256, 152 * 16), 256, 0, st>>>(pairs, rows, nrows,
                                                                                                    rows_per_cell);
}

cudaError_t oz_rank1_classify(const OzNet &net, const Arena &ar, int64_t p0, int64_t p1, int64_t c_begin,
                              int max_chain, R1Scratch &r, cudaStream_t st)
{
    R1Rows rr{};
    for (int l = 1; l <= net.L; ++l) rr.row0[l] = net.row0[l];
    rr.row0[net.L + 1] = net.N;
    cudaError_t e = cudaMemsetAsync(r.counts, 0, sizeof(unsigned long long) * (kMaxLayers + 1), st);
    if (e != cudaSuccess) return e;
    oz_r1_classify_kernel<<<152 * 4, 256, 0, st>>>(ar, p0, p1, c_begin, max_chain, net.L, rr, r.counts);
    return cudaGetLastError();
}

cudaError_t oz_rank1_scatter(const Arena &ar, int64_t c0, int64_t c1, const int *h_offs, int L, R1Scratch &r,
                             cudaStream_t st)
{
    (void)L;
    cudaError_t e = cudaMemcpyAsync(r.offs, h_offs, sizeof(int) * 2 * (kMaxLayers + 1), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    const int64_t n = c1 - c0;
    if (n <= 0) return cudaSuccess;
    oz_r1_scatter_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(ar, c0, c1, r.full_list,
                                                                                                  r.r1_list, r.offs);
    return cudaGetLastError();
}

cudaError_t oz_rank1(const OzNet &net, const R1Cells &cells, const int32_t *list, int64_t n, const int64_t *cnt_le,
                     const void *prev_rows, int64_t prev0, void *rows, int64_t cell0, const OzScratch &scr,
                     R1Scratch &r, int tile_cells, int sms, cudaStream_t st)
{
    const int64_t cap = 4 * scr.batch_cells;              // one operand column per child
    const int64_t rstride = 8 * (int64_t)(net.N + 1);
    for (int64_t b0 = 0; b0 < n; b0 += cap) {
        const int64_t nb = std::min<int64_t>(cap, n - b0);
        auto le = [&](int x) {                            // children of this batch with flip layer <= x
            const int64_t v = x < 1 ? 0 : cnt_le[x] - b0;
            return std::max<int64_t>(0, std::min<int64_t>(nb, v));
        };
        R1Init in{};
        in.keys = cells.keys;
        in.kw = cells.kw;
        in.list = list + b0;
        in.parent = cells.parent;
        in.entry = cells.entry;
        in.prev_rows = reinterpret_cast<const float *>(prev_rows);
        in.prev0 = prev0;
        in.rows = reinterpret_cast<float *>(rows);
        in.cell0 = cell0;
        in.rstride = rstride;
        in.L = net.L;
        in.N = net.N;
        for (int l = 1; l <= net.L; ++l) in.row0[l] = net.row0[l];
        in.row0[net.L + 1] = net.N;
        in.w_out = net.w_out;
        in.it_l = r.it_l;
        in.it_k = r.it_k;
        in.it_a = r.it_a;
        oz_r1_init_kernel<<<(unsigned)nb, 128, 0, st>>>(in);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        for (int j = 2; j <= net.L; ++j) {
            const int64_t g = le(j - 2), pc = le(j - 1);
            int zero = 0;
            if (g > 0) {
                e = oz_layer_product(net, j, scr, g, tile_cells, sms, st, &zero);
                if (e != cudaSuccess) return e;
            }
            if (pc == 0) continue;
            R1Prep pp{};
            pp.keys = cells.keys;
            pp.kw = cells.kw;
            pp.list = list + b0;
            pp.parent = cells.parent;
            pp.prev_rows = reinterpret_cast<const float *>(prev_rows);
            pp.prev0 = prev0;
            pp.rows = reinterpret_cast<float *>(rows);
            pp.cell0 = cell0;
            pp.rstride = rstride;
            pp.j = j;
            pp.L = net.L;
            pp.N = net.N;
            pp.nj = net.width[j];
            pp.row0j = net.row0[j];
            pp.ATj = net.AT[j];
            pp.eA = net.eA[j];
            pp.P = scr.P;
            pp.Q = scr.Q;
            pp.zero = zero;
            pp.Mp = oz_mp(net.width[j]);
            pp.eBin = scr.eB[j & 1];
            pp.eBout = scr.eB[(j + 1) & 1];
            pp.B = scr.B;
            pp.ncols = 4 * scr.batch_cells;
            pp.Kp = oz_kp(net.width[j]);
            pp.w_out = net.w_out;
            pp.it_l = r.it_l;
            pp.it_k = r.it_k;
            pp.it_a = r.it_a;
            oz_r1_prep_kernel<<<(unsigned)pc, kOzPrepThreads, 2 * sizeof(float) * net.width[j], st>>>(pp);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace am
