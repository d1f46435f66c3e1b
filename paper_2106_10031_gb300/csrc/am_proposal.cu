// am_proposal.cu -- the learned constraint proposal: a small MLP, trained on the GPU, that
// scores every hidden neuron of the meshed net by how likely its plane carries an edge of a
// cell's face.  The march clips with its 32 best-scored rows first; the all-row check that
// follows keeps the mesh exact whatever the scores are.
//
//   x (7 + L) -> h1 = relu(W1 x + b1) (H) -> h2 = relu(W2 h1 + b2) (H) -> z = W3 h2 + b3 (n_out)
//   training loss: mean binary cross-entropy of sigmoid(z) against the 0/1 boundary labels.
//
// Training is mixed precision: FP32 master weights, BF16 operands for every matrix product,
// FP32 accumulation, Adam.  Matrix products use one tiled kernel (64 x 64 output tile per
// block, 16-deep K slices staged in shared memory).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cuda_bf16.h>
#include <vector>

#include "am_kernels.h"

namespace am {

constexpr int kGT = 64;     // GEMM output tile
constexpr int kGK = 16;     // GEMM K slice

// C[M x N] = alpha * op(A)[M x K] * op(B)[K x N] + beta * C.  A is row-major M x K (lda = K) or,
// with ta, stored K x M (lda = M); B is row-major K x N (ldb = N) or, with tb, stored N x K.
__global__ void __launch_bounds__(256) gemm_bf16_kernel(int M, int N, int K, const __nv_bfloat16 *A, int lda,
                                                        bool ta, const __nv_bfloat16 *B, int ldb, bool tb, float *C,
                                                        int ldc, float alpha, float beta)
{
    __shared__ float As[kGK][kGT + 1];
    __shared__ float Bs[kGK][kGT + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int row0 = blockIdx.y * kGT, col0 = blockIdx.x * kGT;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += kGK) {
        for (int i = threadIdx.x; i < kGK * kGT; i += 256) {
            const int kk = i / kGT, mm = i % kGT;
            const int gr = row0 + mm, gk = k0 + kk;
            float va = 0.0f, vb = 0.0f;
            if (gr < M && gk < K) va = __bfloat162float(ta ? A[(size_t)gk * lda + gr] : A[(size_t)gr * lda + gk]);
            const int gc = col0 + mm;
            if (gc < N && gk < K) vb = __bfloat162float(tb ? B[(size_t)gc * ldb + gk] : B[(size_t)gk * ldb + gc]);
            As[kk][mm] = va;
            Bs[kk][mm] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty + 16 * i]; b[i] = Bs[kk][tx + 16 * i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
            if (r < M && c < N) {
                float *p = C + (size_t)r * ldc + c;
                *p = alpha * acc[i][j] + (beta != 0.0f ? beta * *p : 0.0f);
            }
        }
}

static void gemm(int M, int N, int K, const __nv_bfloat16 *A, int lda, bool ta, const __nv_bfloat16 *B, int ldb,
                 bool tb, float *C, int ldc, float alpha, float beta, cudaStream_t st)
{
    dim3 grid((N + kGT - 1) / kGT, (M + kGT - 1) / kGT);
    gemm_bf16_kernel<<<grid, 256, 0, st>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, alpha, beta);
}

__global__ void to_bf16_kernel(const float *x, __nv_bfloat16 *y, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// Z (rows x cols) += bias; H = relu(Z) in BF16 (pre-activations kept for the backward pass)
__global__ void bias_relu_kernel(float *Z, const float *b, __nv_bfloat16 *H, int rows, int cols, int relu)
{
    const int64_t n = (int64_t)rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float z = Z[i] + b[i % cols];
        Z[i] = z;
        if (H) H[i] = __float2bfloat16_rn(relu ? fmaxf(z, 0.0f) : z);
    }
}

// dZ = (sigmoid(z) - y) / (rows cols) in BF16; per-block partial sums of softplus(z) - y z
__global__ void bce_kernel(const float *Z, const float *Y, __nv_bfloat16 *dZ, float *dZf, int64_t n, float scale,
                           float *loss_parts)
{
    __shared__ float red[256];
    float acc = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float z = Z[i], y = Y[i];
        const float sp = z > 0.0f ? z + log1pf(expf(-z)) : log1pf(expf(z));
        acc += sp - y * z;
        const float g = (1.0f / (1.0f + expf(-z)) - y) * scale;
        dZ[i] = __float2bfloat16_rn(g);
        if (dZf) dZf[i] = g;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_parts[blockIdx.x] = red[0];
}

// dA = dH * (A > 0) (FP32 in, BF16 and FP32 out)
__global__ void relu_back_kernel(const float *dH, const float *A, __nv_bfloat16 *dA, float *dAf, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float g = A[i] > 0.0f ? dH[i] : 0.0f;
        dA[i] = __float2bfloat16_rn(g);
        dAf[i] = g;
    }
}

// db[c] = sum over rows of G[r, c]
__global__ void colsum_kernel(const float *G, int rows, int cols, float *db)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (int r = 0; r < rows; ++r) s += G[(size_t)r * cols + c];
    db[c] = s;
}

// Adam (Kingma & Ba 2015) on the FP32 master weights, then the BF16 copy
__global__ void adam_kernel(float *w, const float *g, float *m, float *v, __nv_bfloat16 *wb, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16_rn(wi);
    }
}

// transposed BF16 copy of a rows x cols FP32 matrix with row stride ld >= rows (the padding is
// zero), for coalesced BF16-pair reads in the march
__global__ void transpose_bf16_kernel(const float *W, int rows, int cols, int ld, __nv_bfloat16 *WT)
{
    const int64_t n = (int64_t)ld * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / ld), r = (int)(i % ld);
        WT[i] = __float2bfloat16_rn(r < rows ? W[(size_t)r * cols + c] : 0.0f);
    }
}

// One warp per face.  The face plane comes from the vertices (Newell's normal, which points
// along +grad F because faces are stored CCW about it); the march computes the same plane from
// a_F, so both give one feature vector up to rounding.
__global__ void __launch_bounds__(256) proposal_samples_kernel(SampleArgs a)
{
    __shared__ float feat[8][7 + kMaxLayers];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < a.nf; i += warps) {
        const int64_t f = a.f0 + i;
        const int64_t cb = a.coff[f] - a.c0;
        if (cb >= a.max_samples) continue;
        const int m = (int)(a.coff[f + 1] - a.coff[f]);
        const int64_t cell = a.perm[f];
        const double *V = a.ar.verts + cell * a.ar.maxv * 3;
        const int32_t *E = a.ar.edges + cell * a.ar.maxv;
        double nx = 0.0, ny = 0.0, nz = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
        for (int j = 0; j < m; ++j) {
            const double *p = V + 3 * j, *q = V + 3 * ((j + 1) % m);
            nx += p[1] * q[2] - p[2] * q[1];
            ny += p[2] * q[0] - p[0] * q[2];
            nz += p[0] * q[1] - p[1] * q[0];
            cx += p[0]; cy += p[1]; cz += p[2];
        }
        const double inv = 1.0 / sqrt(nx * nx + ny * ny + nz * nz);
        nx *= inv; ny *= inv; nz *= inv;
        const double off = -(nx * cx + ny * cy + nz * cz) / m;
        float *x = feat[threadIdx.x >> 5];
        if (lane < a.L) {
            const unsigned long long *key = a.ar.keys + cell * a.ar.kw;
            const int r0 = a.row0[lane + 1], n = a.width[lane + 1];
            int cnt = 0;
            for (int b = r0; b < r0 + n; ++b) cnt += (int)((key[b >> 6] >> (b & 63)) & 1ull);
            x[7 + lane] = (float)cnt / (float)n;
        }
        if (lane == 0) { x[3] = (float)nx; x[4] = (float)ny; x[5] = (float)nz; x[6] = (float)off; }
        for (int j = 0; j < m && cb + j < a.max_samples; ++j) {
            const int64_t smp = cb + j;
            const double *p = V + 3 * j, *q = V + 3 * ((j + 1) % m);
            if (lane < 3) x[lane] = (float)(0.5 * (p[lane] + q[lane]));
            __syncwarp();
            for (int c = lane; c < a.n_in; c += 32) a.X[smp * a.n_in + c] = x[c];
            __syncwarp();
            float *y = a.Y + smp * a.N;
            for (int k = lane; k < a.N; k += 32) y[k] = 0.0f;
            __syncwarp();
            for (int t = lane; t < m; t += 32)
                if (E[t] < a.N) y[E[t]] = 1.0f;
            __syncwarp();
        }
    }
}

void launch_proposal_samples(const SampleArgs &a, cudaStream_t st)
{
    const int64_t blocks = std::min<int64_t>((a.nf + 7) / 8, 152 * 8);
    if (blocks > 0) proposal_samples_kernel<<<(int)blocks, 256, 0, st>>>(a);
}

static int blocks_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

// ------------------------------------------------------------------------------------------

cudaError_t proposal_alloc(ProposalDev &p, int n_in, int hidden, int n_out, int max_batch)
{
    p.n_in = n_in;
    p.hidden = hidden;
    p.n_out = n_out;
    p.max_batch = max_batch;
    const int64_t sizes[6] = {(int64_t)hidden * n_in, hidden, (int64_t)hidden * hidden, hidden, (int64_t)n_out * hidden,
                              n_out};
    int64_t tot = 0;
    for (int i = 0; i < 6; ++i) { p.off[i] = tot; tot += sizes[i]; }
    p.off[6] = tot;
    p.n_params = tot;
    cudaError_t e;
    if ((e = cudaMalloc(&p.w, sizeof(float) * tot))) return e;
    if ((e = cudaMalloc(&p.g, sizeof(float) * tot))) return e;
    if ((e = cudaMalloc(&p.m, sizeof(float) * tot))) return e;
    if ((e = cudaMalloc(&p.v, sizeof(float) * tot))) return e;
    if ((e = cudaMalloc(&p.wb, sizeof(__nv_bfloat16) * tot))) return e;
    if ((e = cudaMalloc(&p.w2t, sizeof(__nv_bfloat16) * hidden * hidden))) return e;
    if ((e = cudaMalloc(&p.w3t, sizeof(__nv_bfloat16) * hidden * (n_out + 1)))) return e;
    const int64_t act = (int64_t)max_batch * std::max(std::max(hidden, n_out), n_in);
    for (int i = 0; i < 8; ++i)
        if ((e = cudaMalloc(&p.buf[i], sizeof(float) * act))) return e;
    for (int i = 0; i < 4; ++i)
        if ((e = cudaMalloc(&p.bbuf[i], sizeof(__nv_bfloat16) * act))) return e;
    if ((e = cudaMalloc(&p.loss_parts, sizeof(float) * 152 * 16))) return e;
    // the forward pass of whole batches on the tensor cores (inference: am_proposal_forward and
    // the level march), when the shape allows it; W2 and W3 are read in place from the BF16 copy
    return prop_tc_alloc(p.tc, n_in, hidden, n_out, std::max(max_batch, 4096), p.wb + p.off[2], p.wb + p.off[4]);
}

void proposal_free(ProposalDev &p)
{
    void *b[] = {p.w, p.g, p.m, p.v, p.wb, p.w2t, p.w3t, p.loss_parts};
    for (void *x : b)
        if (x) cudaFree(x);
    for (int i = 0; i < 8; ++i)
        if (p.buf[i]) cudaFree(p.buf[i]);
    for (int i = 0; i < 4; ++i)
        if (p.bbuf[i]) cudaFree(p.bbuf[i]);
    prop_tc_free(p.tc);
    p = ProposalDev{};
}

void proposal_sync_copies(ProposalDev &p, cudaStream_t st)
{
    to_bf16_kernel<<<blocks_for(p.n_params), 256, 0, st>>>(p.w, p.wb, p.n_params);
    const int ld3 = (p.n_out + 1) & ~1;
    transpose_bf16_kernel<<<blocks_for((int64_t)p.hidden * p.hidden), 256, 0, st>>>(p.w + p.off[2], p.hidden, p.hidden,
                                                                                   p.hidden, p.w2t);
    transpose_bf16_kernel<<<blocks_for((int64_t)ld3 * p.hidden), 256, 0, st>>>(p.w + p.off[4], p.n_out, p.hidden, ld3,
                                                                              p.w3t);
    prop_tc_sync_weights(p.tc, p.w + p.off[0], st);
}

// Forward pass over B samples (B <= max_batch).  Activations: buf0 a1, buf1 a2, buf2 z (FP32);
// bbuf0 x, bbuf1 h1, bbuf2 h2 (BF16).
static void forward(ProposalDev &p, const float *X, int B, cudaStream_t st)
{
    const int H = p.hidden, I = p.n_in, O = p.n_out;
    const __nv_bfloat16 *W1 = p.wb + p.off[0], *W2 = p.wb + p.off[2], *W3 = p.wb + p.off[4];
    to_bf16_kernel<<<blocks_for((int64_t)B * I), 256, 0, st>>>(X, p.bbuf[0], (int64_t)B * I);
    gemm(B, H, I, p.bbuf[0], I, false, W1, I, true, p.buf[0], H, 1.0f, 0.0f, st);          // a1 = X W1^T
    bias_relu_kernel<<<blocks_for((int64_t)B * H), 256, 0, st>>>(p.buf[0], p.w + p.off[1], p.bbuf[1], B, H, 1);
    gemm(B, H, H, p.bbuf[1], H, false, W2, H, true, p.buf[1], H, 1.0f, 0.0f, st);          // a2 = h1 W2^T
    bias_relu_kernel<<<blocks_for((int64_t)B * H), 256, 0, st>>>(p.buf[1], p.w + p.off[3], p.bbuf[2], B, H, 1);
    gemm(B, O, H, p.bbuf[2], H, false, W3, H, true, p.buf[2], O, 1.0f, 0.0f, st);          // z = h2 W3^T
    bias_relu_kernel<<<blocks_for((int64_t)B * O), 256, 0, st>>>(p.buf[2], p.w + p.off[5], nullptr, B, O, 0);
}

// Loss and gradients (into p.g) over B samples; returns the number of loss partial blocks.
static int backward(ProposalDev &p, const float *Y, int B, cudaStream_t st)
{
    const int H = p.hidden, I = p.n_in, O = p.n_out;
    const int64_t nz = (int64_t)B * O;
    const int nb = blocks_for(nz);
    // dz (BF16 in bbuf3, FP32 in buf3)
    bce_kernel<<<nb, 256, 0, st>>>(p.buf[2], Y, p.bbuf[3], p.buf[3], nz, 1.0f / (float)nz, p.loss_parts);
    gemm(O, H, B, p.bbuf[3], O, true, p.bbuf[2], H, false, p.g + p.off[4], H, 1.0f, 0.0f, st);   // dW3 = dz^T h2
    colsum_kernel<<<(O + 255) / 256, 256, 0, st>>>(p.buf[3], B, O, p.g + p.off[5]);
    gemm(B, H, O, p.bbuf[3], O, false, p.wb + p.off[4], H, false, p.buf[4], H, 1.0f, 0.0f, st); // dh2 = dz W3
    relu_back_kernel<<<blocks_for((int64_t)B * H), 256, 0, st>>>(p.buf[4], p.buf[1], p.bbuf[3], p.buf[5], (int64_t)B * H);
    gemm(H, H, B, p.bbuf[3], H, true, p.bbuf[1], H, false, p.g + p.off[2], H, 1.0f, 0.0f, st);   // dW2 = da2^T h1
    colsum_kernel<<<(H + 255) / 256, 256, 0, st>>>(p.buf[5], B, H, p.g + p.off[3]);
    gemm(B, H, H, p.bbuf[3], H, false, p.wb + p.off[2], H, false, p.buf[4], H, 1.0f, 0.0f, st); // dh1 = da2 W2
    relu_back_kernel<<<blocks_for((int64_t)B * H), 256, 0, st>>>(p.buf[4], p.buf[0], p.bbuf[3], p.buf[6], (int64_t)B * H);
    gemm(H, I, B, p.bbuf[3], H, true, p.bbuf[0], I, false, p.g + p.off[0], I, 1.0f, 0.0f, st);   // dW1 = da1^T x
    colsum_kernel<<<(H + 255) / 256, 256, 0, st>>>(p.buf[6], B, H, p.g + p.off[1]);
    return nb;
}

cudaError_t proposal_forward(ProposalDev &p, const float *X, int n, float *Z, cudaStream_t st)
{
    if (p.tc.ok) {
        // tensor cores: BF16 operands (features, h1, h2 rounded to BF16 as in training), FP32
        // accumulation, FP32 logits
        for (int s = 0; s < n; s += p.tc.max_rows) {
            const int B = std::min(p.tc.max_rows, n - s);
            cudaError_t e = prop_tc_pack(p.tc, X + (size_t)s * p.n_in, B, st);
            if (e) return e;
            e = prop_tc_forward(p.tc, p.w + p.off[1], p.w + p.off[3], p.w + p.off[5], B, Z + (size_t)s * p.n_out, true,
                                p.n_out, p.tc.err, st);
            if (e) return e;
        }
        return cudaGetLastError();
    }
    for (int s = 0; s < n; s += p.max_batch) {
        const int B = std::min(p.max_batch, n - s);
        forward(p, X + (size_t)s * p.n_in, B, st);
        cudaError_t e = cudaMemcpyAsync(Z + (size_t)s * p.n_out, p.buf[2], sizeof(float) * B * p.n_out,
                                        cudaMemcpyDeviceToDevice, st);
        if (e) return e;
    }
    return cudaGetLastError();
}

cudaError_t proposal_grad(ProposalDev &p, const float *X, const float *Y, int n, float *loss, cudaStream_t st)
{
    if (n > p.max_batch) return cudaErrorInvalidValue;
    forward(p, X, n, st);
    const int nb = backward(p, Y, n, st);
    std::vector<float> parts(nb);
    cudaError_t e = cudaMemcpyAsync(parts.data(), p.loss_parts, sizeof(float) * nb, cudaMemcpyDeviceToHost, st);
    if (e) return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    double s = 0.0;
    for (float x : parts) s += x;
    *loss = (float)(s / ((double)n * p.n_out));
    return cudaSuccess;
}

cudaError_t proposal_train(ProposalDev &p, const float *X, const float *Y, int64_t n, int batch, int steps, float lr,
                           float *losses, cudaStream_t st)
{
    if (batch > p.max_batch || batch < 1 || n < batch) return cudaErrorInvalidValue;
    int64_t cursor = 0;
    for (int it = 0; it < steps; ++it) {
        if (cursor + batch > n) cursor = 0;
        float loss = 0.0f;
        cudaError_t e = proposal_grad(p, X + cursor * p.n_in, Y + cursor * p.n_out, batch, &loss, st);
        if (e) return e;
        cursor += batch;
        p.step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.0f - powf(b1, (float)p.step), c2 = 1.0f - powf(b2, (float)p.step);
        adam_kernel<<<blocks_for(p.n_params), 256, 0, st>>>(p.w, p.g, p.m, p.v, p.wb, p.n_params, lr, b1, b2, 1e-8f, c1, c2);
        if (losses) losses[it] = loss;
    }
    proposal_sync_copies(p, st);
    return cudaGetLastError();
}

}  // namespace am
