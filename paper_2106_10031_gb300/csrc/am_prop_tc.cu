// am_prop_tc.cu -- the learned proposal's forward pass for a whole batch of cells on the
// tcgen05 tensor cores (no counterpart in the paper).
//
// The proposal is x (7 + L) -> h1 = relu(W1 x + b1) -> h2 = relu(W2 h1 + b2) -> z = W3 h2 + b3.
// For a batch of cells each layer is one dense product: the cells' activations stacked as the
// rows of A ([cells x K], BF16, K-major) against the layer's weights as B ([n_out x K], BF16,
// K-major: W row-major as stored), FP32 accumulation in TMEM, bias and ReLU fused into the
// epilogue, which writes the next layer's BF16 activations (or the scores).  One CTA computes
// a 128-cell x BN-output tile with the whole K (at most 4 chunks of 64) staged at once by TMA:
// warp 0 loads, warp 1 issues the UMMAs (M = 128, N = BN, K = 16), warps 2..5 drain TMEM.
// Every wait is bounded; on a time-out the CTA raises the error flag, lets its copies and
// products in flight finish, frees TMEM and returns.
#include <algorithm>
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "am_kernels.h"
#include "am_tcgen05.cuh"

namespace am {

namespace {

using namespace tc;

constexpr int kPM = 128;                  // cells per CTA (UMMA M)
constexpr int kPBK = 64;                  // K elements per staged chunk (128 bytes of BF16)
constexpr int kPMaxKC = 4;                // K <= 256
constexpr int kPMaxBN = 256;              // outputs per CTA (UMMA N)
constexpr int kPATile = kPM * 128;        // bytes of one A chunk
constexpr int kPBTile = kPMaxBN * 128;    // bytes reserved per B chunk
constexpr int kPSmem = kPMaxKC * (kPATile + kPBTile) + 64 + 1024;

struct PropGemm {
    const float *bias;     // n_out
    void *out;             // rows x ldo, BF16 or FP32
    int ldo;               // elements
    int rows;              // valid rows (cells) of A
    int n_out;             // valid output columns
    int bn;                // outputs per CTA (multiple of 16, <= 256)
    int kc;                // K chunks of 64
    int relu, out_f32;
    int *err;
};

__global__ void __launch_bounds__(192, 1)
    prop_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, PropGemm g)
{
    extern __shared__ unsigned char prop_smem_raw[];
    const uint32_t raw = smem_u32(prop_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = prop_smem_raw + (base - raw);
    const uint32_t sA = base, sB = base + kPMaxKC * kPATile;
    const uint32_t bars = sB + kPMaxKC * kPBTile;
    const uint32_t full = bars, accfull = bars + 8, drain = bars + 16;
    unsigned char *tail = gbase + (bars - base) + 24;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tail);
    volatile int *abort = reinterpret_cast<volatile int *>(tail + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kPM, n0 = blockIdx.y * g.bn;
    if (threadIdx.x == 0) {
        mbar_init(full, 1);
        mbar_init(accfull, 1);
        mbar_init(drain, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kPMaxBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // the whole K at once: every chunk of A and of B on one barrier
            mbar_expect_tx(full, (uint32_t)(g.kc * (kPATile + g.bn * 128)));
            for (int kc = 0; kc < g.kc; ++kc) {
                tma_load_2d(sA + kc * kPATile, &tmA, kc * kPBK, m0, full);
                tma_load_2d(sB + kc * kPBTile, &tmB, kc * kPBK, n0, full);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            if (!mbar_wait(full, 0, abort, g.err)) {
                // the copies in flight must land before the CTA's shared memory goes away
                mbar_drain(full, 0, kDrainNs);
                umma_commit(drain);                  // nothing issued; the commit still arrives
                mbar_drain(drain, 0, kDrainNs);
            } else {
                tc_fence_after();
                const uint32_t idesc = umma_idesc_bf16(kPM, g.bn);
                for (int kc = 0; kc < g.kc; ++kc) {
                    const uint64_t ad = sw128_desc(sA + kc * kPATile), bd = sw128_desc(sB + kc * kPBTile);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_bf16(tmem, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), idesc,
                                  (kc | kk) != 0 ? 1u : 0u);
                }
                umma_commit(accfull);
            }
        }
    } else {
        // epilogue: warp w drains TMEM lanes 32 (w % 4) .. + 31, one cell (row) per thread
        const int quarter = warp & 3;
        const int row = m0 + quarter * 32 + lane;
        if (mbar_wait(accfull, 0, abort, g.err)) {
            tc_fence_after();
            const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
            for (int c0 = 0; c0 < g.bn; c0 += 32) {
                uint32_t v[4][8];
#pragma unroll
                for (int q = 0; q < 4; ++q) tmem_ld8_nowait(trow + (uint32_t)(c0 + 8 * q), v[q]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row >= g.rows) continue;
                float y[32];
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int c = n0 + c0 + 8 * q + j;
                        float a = __uint_as_float(v[q][j]) + (c < g.n_out ? g.bias[c] : 0.0f);
                        y[8 * q + j] = g.relu ? fmaxf(a, 0.0f) : a;
                    }
                const int cbase = n0 + c0;
                if (g.out_f32) {
                    float *o = reinterpret_cast<float *>(g.out) + (int64_t)row * g.ldo + cbase;
                    if (cbase + 32 <= g.n_out) {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            reinterpret_cast<float4 *>(o)[q] = make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
                    } else {
                        for (int j = 0; j < 32 && cbase + j < g.n_out; ++j) o[j] = y[j];
                    }
                } else {
                    __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(g.out) + (int64_t)row * g.ldo + cbase;
                    if (cbase + 32 <= g.n_out) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            uint4 w;
                            unsigned *wp = &w.x;
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                const __nv_bfloat162 b2 = __floats2bfloat162_rn(y[8 * q + 2 * h], y[8 * q + 2 * h + 1]);
                                wp[h] = *reinterpret_cast<const unsigned *>(&b2);
                            }
                            reinterpret_cast<uint4 *>(o)[q] = w;
                        }
                    } else {
                        for (int j = 0; j < 32 && cbase + j < g.n_out; ++j) o[j] = __float2bfloat16_rn(y[j]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPMaxBN) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode_p = nullptr;

cudaError_t encode(CUtensorMap *m, const void *ptr, int64_t K, int64_t rows, int box_rows)
{
    if (!g_encode_p) {
        cudaDriverEntryPointQueryResult q{};
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        g_encode_p = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kPBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode_p(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int out_tile(int n) { return n <= kPMaxBN ? n : kPMaxBN; }

cudaError_t gemm(const CUtensorMap &A, const CUtensorMap &B, int rows, int K, int n_out, const float *bias, void *out,
                 int ldo, bool relu, bool f32, int *err, cudaStream_t st)
{
    PropGemm g{};
    g.bias = bias;
    g.out = out;
    g.ldo = ldo;
    g.rows = rows;
    g.n_out = n_out;
    g.bn = out_tile(n_out);
    g.kc = K / kPBK;
    g.relu = relu ? 1 : 0;
    g.out_f32 = f32 ? 1 : 0;
    g.err = err;
    const dim3 grid((unsigned)((rows + kPM - 1) / kPM), (unsigned)((n_out + g.bn - 1) / g.bn));
    prop_gemm_kernel<<<grid, 192, kPSmem, st>>>(A, B, g);
    return cudaGetLastError();
}

// FP32 samples (rows x n_in) -> BF16 rows of kPBK, zero padded (the A operand of layer 1)
__global__ void prop_pack_kernel(const float *X, int rows, int n_in, __nv_bfloat16 *Xp)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)rows * kPBK;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / kPBK), c = (int)(i % kPBK);
        Xp[i] = __float2bfloat16_rn(c < n_in ? X[(int64_t)r * n_in + c] : 0.0f);
    }
}

// W1 (hidden x n_in, FP32 master) -> BF16 hidden x kPBK, zero padded
__global__ void prop_pad_w1_kernel(const float *W1, int hidden, int n_in, __nv_bfloat16 *W1p)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < hidden * kPBK; i += gridDim.x * blockDim.x) {
        const int r = i / kPBK, c = i % kPBK;
        W1p[i] = __float2bfloat16_rn(c < n_in ? W1[r * n_in + c] : 0.0f);
    }
}

// Features of the cells [c0, c0 + n) of the level march, one warp per cell, in the layout the
// in-march proposal uses: entry point (3), unit normal of a_F (3), a_F offset / |normal| (1),
// active fraction of each hidden layer (L), zero padded to kPBK BF16 values.  a_F is row N of
// the cell's composed rows (FP32 pairs: the hi words [hi x 4] of rows 0..N, then their lo words).
__global__ void prop_features_kernel(PropFeatures f)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= f.n) return;
    const int64_t cell = f.c0 + i;
    // the unit face plane in FP32 from the hi and lo words of a_F: the features are BF16 (8
    // bits), so FP32 carries them with room to spare, and this part's FP64 pipe is narrow
    const float *aF = f.rows + i * f.rstride + 4 * (int64_t)f.N;             // hi words of a_F
    const float *aL = f.rows + i * f.rstride + 4 * (int64_t)(2 * f.N + 1);   // its lo words
    const float F0 = aF[0] + aL[0], F1 = aF[1] + aL[1], F2 = aF[2] + aL[2], F3 = aF[3] + aL[3];
    const float inv = rsqrtf(F0 * F0 + F1 * F1 + F2 * F2);
    __nv_bfloat16 *o = f.X + i * kPBK;
    for (int j = lane; j < kPBK; j += 32) {
        float x = 0.0f;
        if (j < 3) x = f.entry_pt[cell * 3 + j];
        else if (j == 3) x = (float)(F0 * inv);
        else if (j == 4) x = (float)(F1 * inv);
        else if (j == 5) x = (float)(F2 * inv);
        else if (j == 6) x = (float)(F3 * inv);
        else if (j < 7 + f.L) {
            const int l = j - 6;
            const int r0 = f.row0[l], n = f.width[l];
            const unsigned long long *key = f.keys + cell * f.kw;
            int cnt = 0;
            for (int w = r0 >> 6; w <= (r0 + n - 1) >> 6; ++w) {
                unsigned long long bits = key[w];
                const int lo = max(r0 - 64 * w, 0), hi = min(r0 + n - 64 * w, 64);
                const unsigned long long mhi = hi >= 64 ? ~0ull : ((1ull << hi) - 1ull);
                bits &= mhi & ~((1ull << lo) - 1ull);
                cnt += __popcll(bits);
            }
            x = (float)cnt / (float)n;
        }
        o[j] = __float2bfloat16_rn(x);
    }
}

}  // namespace

bool prop_tc_shape_ok(int n_in, int hidden, int n_out)
{
    return n_in >= 1 && n_in <= kPBK && hidden % kPBK == 0 && hidden <= kPMaxKC * kPBK && n_out >= 16 &&
           n_out % 16 == 0 && (n_out <= kPMaxBN || n_out % kPMaxBN == 0);
}

cudaError_t prop_tc_alloc(PropTC &t, int n_in, int hidden, int n_out, int max_rows, const __nv_bfloat16 *W2,
                          const __nv_bfloat16 *W3)
{
    t = PropTC{};
    if (!prop_tc_shape_ok(n_in, hidden, n_out)) return cudaSuccess;      // t.ok stays false
    cudaError_t e;
    t.max_rows = max_rows;
    if ((e = cudaMalloc(&t.X, sizeof(__nv_bfloat16) * (size_t)max_rows * kPBK))) return e;
    if ((e = cudaMalloc(&t.H1, sizeof(__nv_bfloat16) * (size_t)max_rows * hidden))) return e;
    if ((e = cudaMalloc(&t.H2, sizeof(__nv_bfloat16) * (size_t)max_rows * hidden))) return e;
    if ((e = cudaMalloc(&t.W1p, sizeof(__nv_bfloat16) * (size_t)hidden * kPBK))) return e;
    if ((e = cudaMalloc(&t.scores, sizeof(__nv_bfloat16) * (size_t)max_rows * n_out))) return e;
    if ((e = cudaMalloc(&t.err, sizeof(int)))) return e;
    if ((e = cudaMemset(t.err, 0, sizeof(int)))) return e;
    if ((e = cudaFuncSetAttribute(prop_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmem))) return e;
    auto *m = reinterpret_cast<CUtensorMap *>(t.maps);
    if ((e = encode(&m[0], t.X, kPBK, max_rows, kPM))) return e;
    if ((e = encode(&m[1], t.H1, hidden, max_rows, kPM))) return e;
    if ((e = encode(&m[2], t.H2, hidden, max_rows, kPM))) return e;
    if ((e = encode(&m[3], t.W1p, kPBK, hidden, out_tile(hidden)))) return e;
    if ((e = encode(&m[4], W2, hidden, hidden, out_tile(hidden)))) return e;
    if ((e = encode(&m[5], W3, hidden, n_out, out_tile(n_out)))) return e;
    t.n_in = n_in;
    t.hidden = hidden;
    t.n_out = n_out;
    t.ok = true;
    return cudaSuccess;
}

void prop_tc_free(PropTC &t)
{
    for (void *p : {(void *)t.X, (void *)t.H1, (void *)t.H2, (void *)t.W1p, (void *)t.scores, (void *)t.err})
        if (p) cudaFree(p);
    t = PropTC{};
}

cudaError_t prop_tc_grow(PropTC &t, int rows)
{
    if (!t.ok || rows <= t.max_rows) return cudaSuccess;
    const int cap = ((rows + rows / 4 + kPM - 1) / kPM) * kPM;
    for (void *p : {(void *)t.X, (void *)t.H1, (void *)t.H2, (void *)t.scores})
        if (p) cudaFree(p);
    t.X = t.H1 = t.H2 = t.scores = nullptr;
    t.ok = false;
    cudaError_t e;
    if ((e = cudaMalloc(&t.X, sizeof(__nv_bfloat16) * (size_t)cap * kPBK))) return e;
    if ((e = cudaMalloc(&t.H1, sizeof(__nv_bfloat16) * (size_t)cap * t.hidden))) return e;
    if ((e = cudaMalloc(&t.H2, sizeof(__nv_bfloat16) * (size_t)cap * t.hidden))) return e;
    if ((e = cudaMalloc(&t.scores, sizeof(__nv_bfloat16) * (size_t)cap * t.n_out))) return e;
    auto *m = reinterpret_cast<CUtensorMap *>(t.maps);
    if ((e = encode(&m[0], t.X, kPBK, cap, kPM))) return e;
    if ((e = encode(&m[1], t.H1, t.hidden, cap, kPM))) return e;
    if ((e = encode(&m[2], t.H2, t.hidden, cap, kPM))) return e;
    t.max_rows = cap;
    t.ok = true;
    return cudaSuccess;
}

void prop_tc_sync_weights(PropTC &t, const float *W1, cudaStream_t st)
{
    if (!t.ok) return;
    prop_pad_w1_kernel<<<(t.hidden * kPBK + 255) / 256, 256, 0, st>>>(W1, t.hidden, t.n_in, t.W1p);
}

cudaError_t prop_tc_pack(const PropTC &t, const float *X, int rows, cudaStream_t st)
{
    const int64_t n = (int64_t)rows * kPBK;
    prop_pack_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, st>>>(X, rows, t.n_in, t.X);
    return cudaGetLastError();
}

cudaError_t prop_tc_features(const PropTC &t, const PropFeatures &f, cudaStream_t st)
{
    PropFeatures g = f;
    g.X = t.X;
    prop_features_kernel<<<(unsigned)((f.n * 32 + 255) / 256), 256, 0, st>>>(g);
    return cudaGetLastError();
}

cudaError_t prop_tc_forward(const PropTC &t, const float *b1, const float *b2, const float *b3, int rows, void *out,
                            bool out_f32, int ldo, int *err, cudaStream_t st)
{
    const auto *m = reinterpret_cast<const CUtensorMap *>(t.maps);
    cudaError_t e;
    if ((e = gemm(m[0], m[3], rows, kPBK, t.hidden, b1, t.H1, t.hidden, true, false, err, st))) return e;
    if ((e = gemm(m[1], m[4], rows, t.hidden, t.hidden, b2, t.H2, t.hidden, true, false, err, st))) return e;
    return gemm(m[2], m[5], rows, t.hidden, t.n_out, b3, out, ldo, false, out_f32, err, st);
}

}  // namespace am
