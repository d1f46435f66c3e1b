// am_cell.cu -- the per-cell kernel of the FP64 path: one thread block solves one cell.
//
//   a2 compose  : Z_l = W_l diag(s_{l-1}) Z_{l-1} + C_l (Lemma 1, Cor. 1), layer by layer,
//                 only over the active neurons of the previous layer; a_F likewise;
//   a3 rows     : c_k = (1 - 2 s_k) Z_k (Eq. 10), kept in shared memory, plus the box rows;
//   a4 clip     : the face plane a_F [x;1] = 0 (Eq. 12) starts as a square around the box
//                 section and is cut by the deepest-cutting constraint first, until no
//                 constraint cuts it; vertices are always re-solved from their two planes
//                 and the face plane (Eq. 11), never interpolated;
//   a5 checks   : planes within delta of a final vertex are counted as degenerate events;
//   a6 emit     : corners and edge planes to the face arena;
//   a7 march    : each edge on a neuron plane flips that neuron's bit (Alg. 1 step 10) and
//                 pushes the neighbour through the hash table (step 11).
// This is a different clip from the oracle's (which pivots along the polygon, Alg. 2); the
// face it computes is the same set by definition (Eq. 12).
#include "am_block.cuh"
#include "am_kernels.h"

namespace am {

constexpr int kCellThreads = 128;
constexpr int kMaxPoly = 64;      // polygon vertices in flight (max_face_verts + 2 <= 64)

struct CellSmem {                  // byte offsets into dynamic shared memory
    int rows, rnorm, part, pv, pe, cand, act, mask, red, total;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline CellSmem cell_smem_layout(int max_n, int max_w)
{
    CellSmem s;
    const int nr = max_n + kBoxPlanes + kSquarePlanes;
    int o = 0;
    s.rows = o;  o = align16(o + nr * 4 * (int)sizeof(double));
    s.rnorm = o; o = align16(o + nr * (int)sizeof(double));
    s.part = o;  o = align16(o + kCellThreads * 4 * (int)sizeof(double));
    s.pv = o;    o = align16(o + 2 * kMaxPoly * 3 * (int)sizeof(double));
    s.pe = o;    o = align16(o + 2 * kMaxPoly * (int)sizeof(int));
    s.cand = o;  o = align16(o + nr * (int)sizeof(int));
    s.act = o;   o = align16(o + max_w * (int)sizeof(int));
    s.mask = o;  o = align16(o + ((max_n + 31) / 32) * (int)sizeof(unsigned));
    s.red = o;   o = align16(o + 32 * (int)sizeof(double) + 64 * (int)sizeof(int) + 16 * (int)sizeof(double));
    s.total = o;
    return s;
}

int cell_smem_bytes(int max_n, int max_w) { return cell_smem_layout(max_n, max_w).total; }

// Vertex of planes p, q and the face plane f (Eq. 11 with biases): n.x = -d for the three,
// by Cramer's rule with cross products.  Returns false if the system is singular.
__device__ __forceinline__ bool solve_vertex(const double *p, const double *q, const double *f, double *v)
{
    const double cqf0 = q[1] * f[2] - q[2] * f[1], cqf1 = q[2] * f[0] - q[0] * f[2], cqf2 = q[0] * f[1] - q[1] * f[0];
    const double cfp0 = f[1] * p[2] - f[2] * p[1], cfp1 = f[2] * p[0] - f[0] * p[2], cfp2 = f[0] * p[1] - f[1] * p[0];
    const double cpq0 = p[1] * q[2] - p[2] * q[1], cpq1 = p[2] * q[0] - p[0] * q[2], cpq2 = p[0] * q[1] - p[1] * q[0];
    const double det = p[0] * cqf0 + p[1] * cqf1 + p[2] * cqf2;
    if (det == 0.0) return false;
    const double inv = -1.0 / det;
    v[0] = (p[3] * cqf0 + q[3] * cfp0 + f[3] * cpq0) * inv;
    v[1] = (p[3] * cqf1 + q[3] * cfp1 + f[3] * cpq1) * inv;
    v[2] = (p[3] * cqf2 + q[3] * cfp2 + f[3] * cpq2) * inv;
    return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}

__device__ __forceinline__ double plane_dist(const double *r, double rinv, const double *v)
{
    return (r[0] * v[0] + r[1] * v[1] + r[2] * v[2] + r[3]) * rinv;
}

__global__ void __launch_bounds__(kCellThreads) cell_fp64_kernel(CellArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const CellSmem L = cell_smem_layout(a.max_n, a.max_w);
    double *rows = (double *)(smem + L.rows);
    double *rnorm = (double *)(smem + L.rnorm);
    double *part = (double *)(smem + L.part);
    double(*pv)[kMaxPoly][3] = (double(*)[kMaxPoly][3])(smem + L.pv);
    int(*pe)[kMaxPoly] = (int(*)[kMaxPoly])(smem + L.pe);
    int *cand = (int *)(smem + L.cand);
    int *act = (int *)(smem + L.act);
    unsigned *mask = (unsigned *)(smem + L.mask);
    double *red_v = (double *)(smem + L.red);
    int *red_i = (int *)(red_v + 32);
    int *wsum = red_i + 32;
    double *sh = (double *)(wsum + 32);     // 16 doubles of per-cell scalars
    int *shi = (int *)(sh + 12);            // 8 ints

    const Arena &ar = a.ar;
    const int tid = threadIdx.x, T = blockDim.x;

    for (int64_t cell = a.begin + blockIdx.x; cell < a.end; cell += gridDim.x) {
        if (ar.nverts[cell] == -2) continue;             // a duplicate seed id: never solved
        const NetDev &net = a.nets[ar.net[cell]];
        const int N = net.N, NR = N + kBoxPlanes + kSquarePlanes;
        const unsigned long long *key = ar.keys + cell * ar.kw;
        for (int w = tid; w < (N + 31) / 32; w += T)
            mask[w] = (unsigned)(key[w >> 1] >> ((w & 1) * 32));
        __syncthreads();

        // ---- a2/a3: compose, layer 1 is cell independent (Cor. 1, l = 1)
        {
            const int n1 = net.width[1];
            const double *C1 = net.Cl[1];
            for (int k = tid; k < n1; k += T) {
                const double sg = ((mask[k >> 5] >> (k & 31)) & 1u) ? -1.0 : 1.0;
                for (int c = 0; c < 4; ++c) rows[k * 4 + c] = sg * C1[k * 4 + c];
            }
        }
        __syncthreads();
        for (int l = 2; l <= net.L; ++l) {
            const int np = net.width[l - 1], nl = net.width[l], rp = net.row0[l - 1], rl = net.row0[l];
            // active list of layer l-1 (diag(s_{l-1}) selects these rows)
            int nact = 0;
            for (int base = 0; base < np; base += T) {
                const int j = base + tid;
                const int f = (j < np) ? (int)((mask[(rp + j) >> 5] >> ((rp + j) & 31)) & 1u) : 0;
                int tot;
                const int pos = block_scan_excl(f, wsum, &tot);
                if (f) act[nact + pos] = j;
                nact += tot;
            }
            __syncthreads();
            const int S = nl >= T ? 1 : T / nl;          // threads sharing one output row
            const double *AT = net.AT[l], *Cl = net.Cl[l];
            for (int item = tid; item < nl * S; item += T) {
                const int k = item % nl, s = item / nl;
                double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                for (int t = s; t < nact; t += S) {
                    const int j = act[t];
                    const double w = __ldg(AT + (size_t)j * nl + k);
                    const double *z = rows + (rp + j) * 4;   // active: z = -row
                    a0 -= w * z[0]; a1 -= w * z[1]; a2 -= w * z[2]; a3 -= w * z[3];
                }
                if (S == 1) {
                    const double sg = ((mask[(rl + k) >> 5] >> ((rl + k) & 31)) & 1u) ? -1.0 : 1.0;
                    double *r = rows + (rl + k) * 4;
                    r[0] = sg * (a0 + Cl[k * 4 + 0]); r[1] = sg * (a1 + Cl[k * 4 + 1]);
                    r[2] = sg * (a2 + Cl[k * 4 + 2]); r[3] = sg * (a3 + Cl[k * 4 + 3]);
                } else {
                    double *p = part + item * 4;
                    p[0] = a0; p[1] = a1; p[2] = a2; p[3] = a3;
                }
            }
            __syncthreads();
            if (S > 1) {
                for (int k = tid; k < nl; k += T) {
                    double acc[4] = {Cl[k * 4 + 0], Cl[k * 4 + 1], Cl[k * 4 + 2], Cl[k * 4 + 3]};
                    for (int s = 0; s < S; ++s)
                        for (int c = 0; c < 4; ++c) acc[c] += part[(s * nl + k) * 4 + c];
                    const double sg = ((mask[(rl + k) >> 5] >> ((rl + k) & 31)) & 1u) ? -1.0 : 1.0;
                    for (int c = 0; c < 4; ++c) rows[(rl + k) * 4 + c] = sg * acc[c];
                }
                __syncthreads();
            }
        }
        // a_F = w_out^T diag(s_L) Z_L + [0 | b_out]  (Cor. 1, Eq. 8)
        {
            const int nL = net.width[net.L], rL = net.row0[net.L];
            double f0 = 0.0, f1 = 0.0, f2 = 0.0, f3 = 0.0;
            for (int k = tid; k < nL; k += T) {
                if ((mask[(rL + k) >> 5] >> ((rL + k) & 31)) & 1u) {
                    const double w = net.w_out[k], *z = rows + (rL + k) * 4;
                    f0 -= w * z[0]; f1 -= w * z[1]; f2 -= w * z[2]; f3 -= w * z[3];
                }
            }
            f0 = warp_sum(f0); f1 = warp_sum(f1); f2 = warp_sum(f2); f3 = warp_sum(f3);
            if ((tid & 31) == 0) {
                part[(tid >> 5) * 4 + 0] = f0; part[(tid >> 5) * 4 + 1] = f1;
                part[(tid >> 5) * 4 + 2] = f2; part[(tid >> 5) * 4 + 3] = f3;
            }
            __syncthreads();
            if (tid == 0) {
                double F[4] = {0.0, 0.0, 0.0, net.b_out};
                for (int w = 0; w < T / 32; ++w)
                    for (int c = 0; c < 4; ++c) F[c] += part[w * 4 + c];
                for (int c = 0; c < 4; ++c) sh[c] = F[c];
            }
        }
        // box rows, norms
        for (int i = tid; i < kBoxPlanes; i += T) {
            double *r = rows + (N + i) * 4;
            r[0] = r[1] = r[2] = 0.0;
            r[i >> 1] = (i & 1) ? -1.0 : 1.0;
            r[3] = -a.box;
        }
        __syncthreads();

        // ---- a4: plane frame and the initial square (thread 0)
        if (tid == 0) {
            const double *F = sh;
            const double nn = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
            int ok = nn > 0.0;
            if (ok) {
                const double p0[3] = {-F[3] * F[0] / nn, -F[3] * F[1] / nn, -F[3] * F[2] / nn};
                const double inv = 1.0 / sqrt(nn);
                const double n[3] = {F[0] * inv, F[1] * inv, F[2] * inv};
                const double ax = fabs(n[0]), ay = fabs(n[1]), az = fabs(n[2]);
                double e[3] = {0.0, 0.0, 0.0};
                e[(ax <= ay && ax <= az) ? 0 : (ay <= az ? 1 : 2)] = 1.0;
                double u[3] = {n[1] * e[2] - n[2] * e[1], n[2] * e[0] - n[0] * e[2], n[0] * e[1] - n[1] * e[0]};
                const double un = 1.0 / sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                u[0] *= un; u[1] *= un; u[2] *= un;
                const double w[3] = {n[1] * u[2] - n[2] * u[1], n[2] * u[0] - n[0] * u[2], n[0] * u[1] - n[1] * u[0]};
                const double s = 1.01 * 1.7320508075688772 * a.box;
                // square edges: -w side, +u side, +w side, -u side (ids N+6..N+9), CCW about n
                const double dirs[4][3] = {{-w[0], -w[1], -w[2]}, {u[0], u[1], u[2]}, {w[0], w[1], w[2]}, {-u[0], -u[1], -u[2]}};
                for (int i = 0; i < 4; ++i) {
                    double *r = rows + (N + kBoxPlanes + i) * 4;
                    r[0] = dirs[i][0]; r[1] = dirs[i][1]; r[2] = dirs[i][2];
                    r[3] = -(dirs[i][0] * p0[0] + dirs[i][1] * p0[1] + dirs[i][2] * p0[2]) - s;
                }
                const double cu[4] = {-1.0, 1.0, 1.0, -1.0}, cw[4] = {-1.0, -1.0, 1.0, 1.0};
                for (int i = 0; i < 4; ++i) {
                    for (int c = 0; c < 3; ++c) pv[0][i][c] = p0[c] + s * (cu[i] * u[c] + cw[i] * w[c]);
                    pe[0][i] = N + kBoxPlanes + i;
                }
            }
            shi[0] = ok ? 4 : 0;     // polygon size
            shi[1] = 0;              // polygon buffer
            shi[2] = 0;              // failure flag
        }
        __syncthreads();
        for (int k = tid; k < NR; k += T) {
            const double *r = rows + k * 4;
            rnorm[k] = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        }
        __syncthreads();

        // candidates: every neuron and box row with a non-zero normal
        int nc = 0;
        for (int base = 0; base < N + kBoxPlanes; base += T) {
            const int k = base + tid;
            const int f = (k < N + kBoxPlanes && rnorm[k] > 0.0) ? 1 : 0;
            int tot;
            const int pos = block_scan_excl(f, wsum, &tot);
            if (f) cand[nc + pos] = k;
            nc += tot;
        }
        __syncthreads();

        // deepest cut first, until no candidate cuts
        for (int round = 0; round < NR && shi[0] > 0; ++round) {
            const int m = shi[0], buf = shi[1];
            double best = 0.0;
            int bk = -1, kept = 0;
            for (int base = 0; base < nc; base += T) {
                const int idx = base + tid;
                const int k = idx < nc ? cand[idx] : -1;
                double depth = -1.0;
                if (k >= 0) {
                    const double *r = rows + k * 4;
                    const double ri = 1.0 / rnorm[k];
                    for (int i = 0; i < m; ++i) depth = fmax(depth, plane_dist(r, ri, pv[buf][i]));
                }
                const int f = (k >= 0 && depth > a.delta) ? 1 : 0;
                int tot;
                const int pos = block_scan_excl(f, wsum, &tot);
                if (f) {
                    cand[kept + pos] = k;
                    if (bk < 0 || depth > best || (depth == best && k < bk)) { best = depth; bk = k; }
                }
                kept += tot;
            }
            nc = kept;
            double bv;
            int bi;
            block_argmax(best, bk, red_v, red_i, &bv, &bi);
            if (bi < 0) break;
            if (tid == 0) {
                const double *r = rows + bi * 4;
                const double ri = 1.0 / rnorm[bi];
                unsigned long long om = 0ull;
                int nout = 0;
                for (int i = 0; i < m; ++i)
                    if (plane_dist(r, ri, pv[buf][i]) > a.delta) { om |= 1ull << i; ++nout; }
                if (nout == m) {
                    shi[0] = 0;
                } else {
                    int ia = -1, ib = -1;
                    for (int i = 0; i < m; ++i) {
                        const bool o = (om >> i) & 1ull;
                        if (o && !((om >> ((i + m - 1) % m)) & 1ull)) ia = i;
                        if (o && !((om >> ((i + 1) % m)) & 1ull)) ib = i;
                    }
                    if (ia < 0 || ib < 0 || ((ib - ia + m) % m) + 1 != nout) {
                        shi[2] = 1;        // the cut is not a single run: inconsistent polygon
                        shi[0] = 0;
                    } else {
                        const int nb = buf ^ 1;
                        int n2 = 0;
                        for (int i = (ib + 1) % m; i != ia; i = (i + 1) % m) {
                            pv[nb][n2][0] = pv[buf][i][0]; pv[nb][n2][1] = pv[buf][i][1]; pv[nb][n2][2] = pv[buf][i][2];
                            pe[nb][n2] = pe[buf][i];
                            ++n2;
                        }
                        const int ea = pe[buf][(ia + m - 1) % m], eb = pe[buf][ib];
                        bool ok = n2 + 2 <= kMaxPoly;
                        if (ok) {
                            ok = solve_vertex(rows + ea * 4, r, sh, pv[nb][n2]);
                            pe[nb][n2] = bi;
                            ok = ok && solve_vertex(r, rows + eb * 4, sh, pv[nb][n2 + 1]);
                            pe[nb][n2 + 1] = eb;
                        }
                        if (!ok) { shi[2] = 2; shi[0] = 0; }
                        else { shi[0] = n2 + 2; shi[1] = nb; }
                    }
                }
            }
            // the applied plane no longer cuts: drop it from the candidates
            __syncthreads();
            for (int idx = tid; idx < nc; idx += T)
                if (cand[idx] == bi) cand[idx] = -1;
            __syncthreads();
            int nn2 = 0;
            for (int base = 0; base < nc; base += T) {
                const int idx = base + tid;
                const int k = idx < nc ? cand[idx] : -1;
                int tot;
                const int pos = block_scan_excl(k >= 0 ? 1 : 0, wsum, &tot);
                if (k >= 0) cand[nn2 + pos] = k;
                nn2 += tot;
            }
            nc = nn2;
            __syncthreads();
        }

        // ---- a5: validity / degeneracy, area, then a6 emit and a7 march
        const int m = shi[0], buf = shi[1];
        int status = shi[2];
        if (m > 0) {
            // a square edge surviving means the plane misses the box interior
            for (int i = 0; i < m; ++i)
                if (pe[buf][i] >= N + kBoxPlanes) status = 3;
        }
        int emit = (m >= 3 && status == 0) ? m : 0;
        if (emit) {
            int nd = 0;
            for (int k = tid; k < N + kBoxPlanes; k += T) {
                if (rnorm[k] == 0.0) continue;
                const double *r = rows + k * 4;
                const double ri = 1.0 / rnorm[k];
                for (int i = 0; i < m; ++i) {
                    const int ea = pe[buf][(i + m - 1) % m], eb = pe[buf][i];
                    if (k == ea || k == eb) continue;
                    if (fabs(plane_dist(r, ri, pv[buf][i])) <= a.delta) ++nd;
                }
            }
            int tot;
            block_scan_excl(nd, wsum, &tot);
            if (tid == 0 && tot) atomicAdd(ar.counters + kDegenerate, (unsigned long long)tot);
            if (tid == 0) {
                double nx = 0.0, ny = 0.0, nz = 0.0;
                for (int i = 0; i < m; ++i) {
                    const double *p = pv[buf][i], *q = pv[buf][(i + 1) % m];
                    nx += p[1] * q[2] - p[2] * q[1]; ny += p[2] * q[0] - p[0] * q[2]; nz += p[0] * q[1] - p[1] * q[0];
                }
                const double area = 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
                shi[3] = area > 1e-24 * a.box * a.box;
            }
            __syncthreads();
            if (!shi[3]) emit = 0;
        }
        if (emit > ar.maxv) {
            if (tid == 0) atomicOr(ar.counters + kStatus, kStFaceVerts);
            emit = 0;
        }
        if (tid == 0) {
            ar.nverts[cell] = emit;
            atomicAdd(ar.counters + kSolved, 1ull);
            if (!emit) atomicAdd(ar.counters + kEmpty, 1ull);
            if (status == 1 || status == 2) atomicOr(ar.counters + kStatus, kStClip);
        }
        if (emit) {
            for (int i = tid; i < m; i += T) {
                ar.edges[cell * ar.maxv + i] = pe[buf][i];
                double *v = ar.verts + (cell * ar.maxv + i) * 3;
                v[0] = pv[buf][i][0]; v[1] = pv[buf][i][1]; v[2] = pv[buf][i][2];
            }
            const unsigned long long h = ar.hash[cell];
            const int nid = ar.net[cell];
            for (int i = tid; i < m; i += T) {
                const int e = pe[buf][i];
                if (e < N) insert_neighbor(ar, cell, nid, (unsigned)e, h ^ ar.zob[e]);
            }
        }
        __syncthreads();
    }
}

void launch_cell_fp64(const CellArgs &a, int grid, cudaStream_t st)
{
    const int smem = cell_smem_bytes(a.max_n, a.max_w);
    cell_fp64_kernel<<<grid, kCellThreads, smem, st>>>(a);
}

cudaError_t prepare_cell_kernels(int max_n, int max_w)
{
    const int smem = cell_smem_bytes(max_n, max_w);
    return cudaFuncSetAttribute(cell_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace am
