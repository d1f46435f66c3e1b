// am_check_tc.cu -- the dense all-constraint check of the sliced level march on the tcgen05
// tensor cores: after the clip, every neuron row of a cell is tested at every vertex of its
// polygon (Eq. 10: the face is the set of points where no row is positive), as one product
// [rows x K] . [K x vertices] per 128-row tile.
//
// Exact operands.  A row's hi word (FP32 per coordinate) is split into three BF16 parts whose
// sum is the word exactly (8 + 8 + 8 significand bits), and so is every vertex coordinate in
// FP32.  K = 16 holds the row's three parts side by side, [r1 | r2 | r3 | 0] (4 coordinates
// each), and the column of vertex i's part q repeats that part three times, [v_q | v_q | v_q |
// 0], so that column's result is r . [v_q; w_q] (w_0 = 1, w_1 = w_2 = 0) with every product
// exact.  Three columns per vertex (parts 1..3, 16 vertices per part) give N = 48.
//
// Certified sign test.  The tensor core adds the 12 exact products of a column in FP32 (at most
// 2^-23 relative per addition, whichever rounding it uses), the three column results are added
// in FP32, the row's lo word and the vertex's rounding to FP32 are left out: the total stays
// below 32 u mag, mag = sum_c |r_c| |v_c| + |r_0| bounded by |r|_1 max_c |v_c| + |r_0| (u = 2^-24).
// With the vertex's own FP64 error (|r|_1 dvb) and the tolerance band delta |r| the test is the
// warp clip's: a row above the bound is violated, a row below minus the bound holds, and a row
// in between is re-evaluated in FP64 from the exact pair.  Any violated row, or a row within the
// band, sends the cell to the block kernel, which solves it with every row (so the mesh is that
// kernel's in every case).
//
// One CTA of 128 threads per record at a time (persistent over the records): thread t stages row
// t of the tile into shared memory in the 128-byte-swizzled K-major layout (only the first 32
// bytes of each 128-byte row are read by a K = 16 product), thread 0 issues the product into
// TMEM, all threads wait on its commit (a bounded wait), and thread t reads TMEM lane t: its own
// row's 48 results.
#include <algorithm>
#include <cuda_bf16.h>

#include "am_common.cuh"
#include "am_kernels.h"
#include "am_tcgen05.cuh"

namespace am {

namespace {

using namespace tc;

constexpr int kCT = 128;                  // threads = rows per tile (UMMA M)
constexpr int kCPart = kChkMaxV;          // columns per vertex part
constexpr int kCN = 3 * kCPart;           // UMMA N
constexpr int kCTmemCols = 64;            // TMEM columns allocated (>= kCN, a power of 2)
constexpr int kCATile = kCT * 128;        // A tile: 128 rows of 128 bytes
constexpr int kCBTile = kCN * 128;        // B tile: 48 rows of 128 bytes
constexpr float kCU = 5.9604645e-8f;      // 2^-24
constexpr float kCBound = 32.0f * kCU;    // the tensor-core evaluation's bound, relative to mag

struct CheckSh {
    double v[kChkMaxV][3];                // FP64 vertices
    float xv[kChkMaxV];                   // max_c |v_c| (FP32 vertex), rounded up
    float dvb[kChkMaxV];                  // bound on each FP64 vertex's error
    float vf[kChkMaxV][3];                // FP32 vertices
    int ea[kChkMaxV], eb[kChkMaxV];       // the two planes of each vertex
    int m;
};

constexpr int kCShOff = kCATile + kCBTile;                     // after the two tiles
// 33 KB per CTA: at most 6 CTAs fit on an SM, so their TMEM (6 x 64 columns) always fits the 512
constexpr int kCSmem = 33 * 1024;
static_assert(1024 + kCShOff + 64 + (int)sizeof(CheckSh) <= kCSmem, "check_tc shared memory");
static_assert((227 * 1024 / kCSmem) * kCTmemCols <= 512, "check_tc TMEM per SM");

// the BF16 parts of x: x = a + b + c exactly (each remainder is exact in FP32 and has at most 8
// significant bits left after two parts)
__device__ __forceinline__ void split3(float x, unsigned &a, unsigned &b, unsigned &c)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    const __nv_bfloat16 l = __float2bfloat16_rn(r2);
    a = __bfloat16_as_ushort(h);
    b = __bfloat16_as_ushort(m);
    c = __bfloat16_as_ushort(l);
}

__device__ __forceinline__ unsigned pack2(unsigned lo, unsigned hi) { return lo | (hi << 16); }

// row `row` of a 128-byte-swizzled K-major tile: 16-byte chunk c of the row at chunk c ^ (row & 7)
__device__ __forceinline__ void st_chunk(unsigned char *tile, int row, int c, uint4 v)
{
    *reinterpret_cast<uint4 *>(tile + row * 128 + ((c ^ (row & 7)) << 4)) = v;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace

__global__ void __launch_bounds__(kCT, 4) check_tc_kernel(CheckArgs a)
{
    extern __shared__ unsigned char chk_smem_raw[];
    const uint32_t raw = smem_u32(chk_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *g = chk_smem_raw + (base - raw);
    unsigned char *tA = g, *tB = g + kCATile;
    const uint32_t sA = base, sB = base + kCATile;
    const uint32_t bar = base + kCShOff;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(g + kCShOff + 8);
    volatile int *abort = reinterpret_cast<volatile int *>(g + kCShOff + 12);
    CheckSh &S = *reinterpret_cast<CheckSh *>(g + kCShOff + 64);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(bar, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    constexpr uint32_t idesc = umma_idesc_bf16(kCT, kCN);

    const int N = a.N;
    const float4 *rows4 = reinterpret_cast<const float4 *>(a.rows);
    const int64_t n_rec = (int64_t)__ldcg(a.count);
    const int ntiles = (N + kCT - 1) / kCT;
    uint32_t phase = 0;
    unsigned long long n_close = 0;
    bool dead = false;
    for (int64_t idx = blockIdx.x; idx < n_rec && !dead; idx += gridDim.x) {
        const CheckRec &R = a.rec[idx];
        const int64_t cell = R.cell;
        const int m = R.m;
        const float4 *rp = rows4 + (cell - a.begin) * 2 * (int64_t)(N + 1);
        // ---- the vertices, and the B tile: row n = 16 q + i holds part q of vertex i
        if (tid < kChkMaxV) {
            const int i = tid;
            if (i < m) {
                const double x = R.v[i][0], y = R.v[i][1], z = R.v[i][2];
                S.v[i][0] = x; S.v[i][1] = y; S.v[i][2] = z;
                const float fx = (float)x, fy = (float)y, fz = (float)z;
                S.vf[i][0] = fx; S.vf[i][1] = fy; S.vf[i][2] = fz;
                S.xv[i] = fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))) * 1.0001f;
                const double X = fmax(1.0, fmax(fabs(x), fmax(fabs(y), fabs(z))));
                S.dvb[i] = (float)(4e-16 * X) * 1.01f;
                S.ea[i] = R.pe[i == 0 ? m - 1 : i - 1];
                S.eb[i] = R.pe[i];
            }
        }
        if (tid == 0) S.m = m;
        if (tid < kCN) {
            const int q = tid / kCPart, i = tid % kCPart;
            unsigned p[4] = {0u, 0u, 0u, 0u};          // BF16 part q of (x, y, z, w)
            if (i < m) {
                unsigned c0, c1, c2;
                const float f[3] = {(float)R.v[i][0], (float)R.v[i][1], (float)R.v[i][2]};
                for (int c = 0; c < 3; ++c) {
                    split3(f[c], c0, c1, c2);
                    p[c] = q == 0 ? c0 : (q == 1 ? c1 : c2);
                }
                p[3] = q == 0 ? 0x3F80u : 0u;          // w: 1 in part 1 only
            }
            const uint4 v01 = make_uint4(pack2(p[0], p[1]), pack2(p[2], p[3]), pack2(p[0], p[1]), pack2(p[2], p[3]));
            const uint4 v2 = make_uint4(pack2(p[0], p[1]), pack2(p[2], p[3]), 0u, 0u);
            st_chunk(tB, tid, 0, v01);
            st_chunk(tB, tid, 1, v2);
        }
        fence_async_smem();
        __syncthreads();
        bool bad = false;
        for (int t = 0; t < ntiles && !dead; ++t) {
            // ---- stage row t kCT + tid: [r1 | r2] in chunk 0, [r3 | 0] in chunk 1
            const int r = t * kCT + tid;
            const float4 h = r < N ? __ldg(rp + r) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            {
                unsigned a0[4], a1[4], a2[4];
                split3(h.x, a0[0], a1[0], a2[0]);
                split3(h.y, a0[1], a1[1], a2[1]);
                split3(h.z, a0[2], a1[2], a2[2]);
                split3(h.w, a0[3], a1[3], a2[3]);
                st_chunk(tA, tid, 0, make_uint4(pack2(a0[0], a0[1]), pack2(a0[2], a0[3]), pack2(a1[0], a1[1]),
                                                pack2(a1[2], a1[3])));
                st_chunk(tA, tid, 1, make_uint4(pack2(a2[0], a2[1]), pack2(a2[2], a2[3]), 0u, 0u));
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                umma_bf16(tmem, sw128_desc(sA), sw128_desc(sB), idesc, 0u);
                umma_commit(bar);
            }
            const bool ok = mbar_wait(bar, phase, abort, a.err);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) { dead = true; break; }
            tc_fence_after();
            uint32_t c[6][8];
#pragma unroll
            for (int q = 0; q < 6; ++q) tmem_ld8_nowait(trow + (uint32_t)(8 * q), c[q]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            // ---- the sign test of row r at every vertex
            const float n2 = h.x * h.x + h.y * h.y + h.z * h.z;
            if (r < N && n2 != 0.0f) {                 // zero normal: a constant row, holds in its own cell
                const float rl1 = fabsf(h.x) + fabsf(h.y) + fabsf(h.z);
                const float band = (float)a.delta * sqrtf(n2) * 1.01f;
#pragma unroll
                for (int i = 0; i < kChkMaxV; ++i) {       // unrolled: the results stay in registers
                    if (i >= m || bad || r == S.ea[i] || r == S.eb[i]) continue;
                    const float s1 = __uint_as_float(c[i >> 3][i & 7]);
                    const float s2 = __uint_as_float(c[2 + (i >> 3)][i & 7]);
                    const float s3 = __uint_as_float(c[4 + (i >> 3)][i & 7]);
                    const float sl = s1 + (s2 + s3);
                    const float mag = __fmaf_ru(rl1, S.xv[i], fabsf(h.w)) * 1.02f;
                    const float B = __fmaf_ru(kCBound, mag, __fmaf_ru(rl1, S.dvb[i], band));
                    if (sl > B) { bad = true; continue; }
                    if (sl >= -B) {                     // close call: FP64 from the exact pair
                        ++n_close;
                        const float4 lo = __ldg(rp + (N + 1) + r);
                        const double r6[4] = {(double)h.x + (double)lo.x, (double)h.y + (double)lo.y,
                                              (double)h.z + (double)lo.z, (double)h.w + (double)lo.w};
                        const double *v6 = S.v[i];
                        const double s6 = r6[0] * v6[0] + r6[1] * v6[1] + r6[2] * v6[2] + r6[3];
                        const double m6 = fabs(r6[0] * v6[0]) + fabs(r6[1] * v6[1]) + fabs(r6[2] * v6[2]) + fabs(r6[3]);
                        const double B6 = (double)rl1 * 1.0001 * (double)S.dvb[i] + (double)band + 1e-15 * m6;
                        if (s6 >= -B6) bad = true;      // violated, or within the band
                    }
                }
            }
            tc_fence_before();
            if (__syncthreads_or(bad)) { bad = true; break; }   // also: TMEM read before the next product
        }
        if (dead) break;
        // ---- the box rows (plane N + i: +x, -x, +y, -y, +z, -z), on the ALU as in the warp clip
        if (!bad && tid < kBoxPlanes) {
            const int i = tid, ax = i >> 1;
            const float sg = (i & 1) ? -1.0f : 1.0f;
            const float rr[4] = {ax == 0 ? sg : 0.0f, ax == 1 ? sg : 0.0f, ax == 2 ? sg : 0.0f, -a.box};
            const float band = (float)a.delta * 1.01f;
            for (int j = 0; j < m; ++j) {
                if (N + i == S.ea[j] || N + i == S.eb[j]) continue;
                const float *v = S.vf[j];
                const float sl = rr[0] * v[0] + rr[1] * v[1] + rr[2] * v[2] + rr[3];
                const float mag = fabsf(rr[0] * v[0]) + fabsf(rr[1] * v[1]) + fabsf(rr[2] * v[2]) + fabsf(rr[3]);
                const float B = __fmaf_ru(8.5f * kCU, mag, __fmaf_ru(1.0f, S.dvb[j], band));
                if (sl > B) { bad = true; break; }
                if (sl >= -B) {
                    ++n_close;
                    const double *v6 = S.v[j];
                    const double s6 = (double)rr[0] * v6[0] + (double)rr[1] * v6[1] + (double)rr[2] * v6[2] + (double)rr[3] -
                                      (double)a.box_lo;
                    const double B6 = 1.0001 * (double)S.dvb[j] + (double)band + 1e-15 * (fabs(v6[ax]) + (double)a.box);
                    if (s6 >= -B6) { bad = true; break; }
                }
            }
        }
        bad = __syncthreads_or(bad);
        if (tid == 0) a.status[idx] = bad ? 1 : 0;
        __syncthreads();                                // the vertex data and B tile are rewritten next
    }
    // ---- teardown: after an abort let the product in flight land (bounded), then free TMEM
    if (__syncthreads_or(dead)) {
        if (tid == 0) {
            mbar_drain(bar, phase ^ 1u, kDrainNs);
        }
    }
    for (int o = 16; o > 0; o >>= 1) n_close += __shfl_xor_sync(0xffffffffu, n_close, o);
    if (lane == 0 && n_close) atomicAdd(a.counters + kCloseCalls, n_close);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCTmemCols) : "memory");
    }
}

cudaError_t prepare_check_tc()
{
    return cudaFuncSetAttribute(check_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCSmem);
}

void launch_check_tc(const CheckArgs &a, int sms, cudaStream_t st)
{
    check_tc_kernel<<<sms * 4, kCT, kCSmem, st>>>(a);
}

}  // namespace am
