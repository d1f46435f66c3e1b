// am_clip_warp.cu -- the clip of the sliced level march with one warp per cell (Alg. 1 steps 6-11
// on rows composed beforehand on the tensor cores).
//
// A block holds kWW warps and each warp solves its own cell start to finish, so the serial
// parts of a cell (the cuts of its polygon) occupy one warp instead of idling a whole block,
// and many cells are in flight per SM.  The rows are read from memory where the block version
// stages them in shared memory: FP32 pairs, a_F last, the cell's N + 1 hi words [hi x 4] and then
// its N + 1 lo words [lo x 4], so a pass that reads only hi words reads half the bytes.  Per cell:
//   candidates : each lane keeps the two rows nearest to the point the cell was entered through
//                among the rows it scans, and with learned candidates also the row the proposal
//                scores highest among them (the proposal extends the nearest set);
//   clip       : the square about the box section is cut by those 64 (96) candidates, nearest cutting
//                row first, in FP32 (Eq. 11 per new vertex), then every vertex is re-solved in
//                FP64 from its two planes;
//   check      : every row at every vertex with a certified FP32 bound; close calls in FP64;
//                violated rows are cut in (FP64) and the check repeats;
//   emit, push : the face record, then each neuron edge pushes its neighbour (Alg. 1 step 10).
// A cell that needs more than this (a test the FP64 close call cannot decide, a row within the
// tolerance band of a vertex, a polygon beyond the warp's capacity, too many violators) is
// handed, untouched, to a list that the block kernel then solves with its FP64 fallback, so the
// result is the block kernel's in every case.
#include <algorithm>
#include <cuda_bf16.h>

#include "am_block.cuh"
#include "am_kernels.h"

namespace am {

namespace {

constexpr int kWW = 8;            // warps (cells) per block
constexpr int kWPoly = 48;        // polygon vertices a warp holds
constexpr int kWViol = 32;        // violated rows cut in per check round
constexpr int kWMaxKw = 128;      // key words (N <= 8190)
constexpr int kWMaxFix = 8;       // check / fix-up rounds
constexpr float kWU = 5.9604645e-8f;   // 2^-24

struct WarpSh {
    double pv[2][kWPoly][3];      // FP64 polygon
    float pf[2][kWPoly][3];       // FP32 polygon of the candidate pass
    int pe[2][kWPoly];            // edge planes (edge i: vertex i -> i + 1)
    float4 vf[kWPoly];            // FP32 vertices (x, y, z) and the vertex term of the check's bound (w)
    int2 ve[kWPoly];              // the planes of the two edges at each vertex
    float dvb[kWPoly];            // bound on each FP64 vertex's error
    float sq[4][4];               // the initial square's rows (planes N + 6 .. N + 9)
    int viol[kWViol];
    double aF[4];
    float aFhi[4];
    int nviol, flag;
    unsigned key[2 * kWMaxKw];    // the cell's key as 32-bit words (pushes copy it)
};

int warp_smem_bytes() { return kWW * (int)sizeof(WarpSh); }

// the rows of one cell: N rows in memory, the 6 box rows and the 4 square rows analytic
struct WRows {
    const float4 *p;              // [hi, lo] per row
    int N;
    float box, box_lo;            // the box as an FP32 pair: box rows' offsets -box (hi), -box_lo (lo)
    const WarpSh *S;
    __device__ __forceinline__ float4 hi(int k) const
    {
        if (k < N) return __ldg(p + k);
        if (k < N + kBoxPlanes) {
            const int i = k - N;
            const float sg = (i & 1) ? -1.0f : 1.0f;
            return make_float4((i >> 1) == 0 ? sg : 0.0f, (i >> 1) == 1 ? sg : 0.0f, (i >> 1) == 2 ? sg : 0.0f, -box);
        }
        const float *q = S->sq[k - N - kBoxPlanes];
        return make_float4(q[0], q[1], q[2], q[3]);
    }
    __device__ __forceinline__ void f64(int k, double *r) const
    {
        const float4 h = hi(k);
        if (k < N) {
            const float4 l = __ldg(p + (N + 1) + k);
            r[0] = (double)h.x + (double)l.x; r[1] = (double)h.y + (double)l.y;
            r[2] = (double)h.z + (double)l.z; r[3] = (double)h.w + (double)l.w;
        } else {
            r[0] = h.x; r[1] = h.y; r[2] = h.z;
            r[3] = k < N + kBoxPlanes ? (double)h.w - (double)box_lo : (double)h.w;
        }
    }
    __device__ __forceinline__ void f32(int k, float *r) const
    {
        const float4 h = hi(k);
        r[0] = h.x; r[1] = h.y; r[2] = h.z; r[3] = h.w;
    }
};

template <class R>
__device__ __forceinline__ R wpdist(const R *r, R ri, const R *v)
{
    return (r[0] * v[0] + r[1] * v[1] + r[2] * v[2] + r[3]) * ri;
}

template <class R>
__device__ __forceinline__ void wrow(const WRows &rv, int k, R *r)
{
    if constexpr (sizeof(R) == 8) rv.f64(k, r);
    else rv.f32(k, r);
}

// One cut of the polygon P[buf] (m vertices) by row k, the warp's lanes over the vertices: a
// vertex is cut off when its distance from row k's plane exceeds tol; the two new vertices are
// solved from their planes and the face plane aF.  Returns the new count (0 = empty, -1 =
// inconsistent or beyond kWPoly); *swapped: the result went to buffer buf ^ 1.
template <class R>
__device__ int wcut(WarpSh &S, R (*P)[kWPoly][3], int m, int buf, int k, R tol, const R *aF, const WRows &rv,
                    bool *swapped)
{
    const int lane = threadIdx.x & 31;
    *swapped = false;
    R rk[4];
    wrow<R>(rv, k, rk);
    const R rn = sqrt(rk[0] * rk[0] + rk[1] * rk[1] + rk[2] * rk[2]);
    if (rn == R(0)) return m;
    const R ri = R(1) / rn;
    const bool o0 = lane < m && wpdist(rk, ri, P[buf][lane]) > tol;
    const bool o1 = lane + 32 < m && wpdist(rk, ri, P[buf][lane + 32]) > tol;
    const unsigned long long out = (unsigned long long)__ballot_sync(0xffffffffu, o0) |
                                   ((unsigned long long)__ballot_sync(0xffffffffu, o1) << 32);
    const int nout = __popcll(out);
    if (nout == 0) return m;
    if (nout == m) return 0;
    int ia = -1, ib = -1;
    for (int i = lane; i < m; i += 32) {
        const bool oi = (out >> i) & 1ull;
        const int ip = i == 0 ? m - 1 : i - 1, in = i + 1 == m ? 0 : i + 1;
        if (oi && !((out >> ip) & 1ull)) ia = i;
        if (oi && !((out >> in) & 1ull)) ib = i;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ia = max(ia, __shfl_xor_sync(0xffffffffu, ia, o));
        ib = max(ib, __shfl_xor_sync(0xffffffffu, ib, o));
    }
    if (ia < 0 || ib < 0 || ((ib - ia + m) % m) + 1 != nout) return -1;
    const int nin = m - nout;
    if (nin + 2 > kWPoly) return -1;
    const int nb = buf ^ 1;
    const int ea = S.pe[buf][ia == 0 ? m - 1 : ia - 1], eb = S.pe[buf][ib];
    for (int i = lane; i < m; i += 32) {                 // the kept run b+1 .. a-1, in order
        if ((out >> i) & 1ull) continue;
        int ni = i - (ib + 1);
        if (ni < 0) ni += m;
        P[nb][ni][0] = P[buf][i][0]; P[nb][ni][1] = P[buf][i][1]; P[nb][ni][2] = P[buf][i][2];
        S.pe[nb][ni] = S.pe[buf][i];
    }
    bool ok = true;
    if (lane < 2) {
        R pa[4], pb[4], v[3];
        wrow<R>(rv, lane == 0 ? ea : k, pa);
        wrow<R>(rv, lane == 0 ? k : eb, pb);
        ok = solve3<R>(pa, pb, aF, v, nullptr);
        P[nb][nin + lane][0] = v[0]; P[nb][nin + lane][1] = v[1]; P[nb][nin + lane][2] = v[2];
        S.pe[nb][nin + lane] = lane == 0 ? k : eb;
    }
    ok = __all_sync(0xffffffffu, ok);
    __syncwarp();
    *swapped = true;
    return ok ? nin + 2 : -1;
}

// the polygon's vertices in FP64 from its planes' rows (exact pairs: no row error term), with
// the bound on their rounding; false when a vertex cannot be solved
__device__ bool wfinal(WarpSh &S, int m, int buf, const WRows &rv)
{
    const int lane = threadIdx.x & 31;
    bool ok = true;
    for (int i = lane; i < m; i += 32) {
        const int ea = S.pe[buf][i == 0 ? m - 1 : i - 1], eb = S.pe[buf][i];
        double ra[4], rb[4], v[3];
        rv.f64(ea, ra);
        rv.f64(eb, rb);
        const bool good = solve3<double>(ra, rb, S.aF, v, nullptr);
        const double X = fmax(1.0, fmax(fabs(v[0]), fmax(fabs(v[1]), fabs(v[2]))));
        S.pv[buf][i][0] = v[0]; S.pv[buf][i][1] = v[1]; S.pv[buf][i][2] = v[2];
        S.dvb[i] = (float)(4e-16 * X) * 1.01f;
        ok = ok && good;
    }
    ok = __all_sync(0xffffffffu, ok);
    __syncwarp();
    return ok;
}

__device__ __forceinline__ unsigned order_key(float d)
{
    const unsigned du = __float_as_uint(d);
    return (du & 0x80000000u) ? ~du : (du | 0x80000000u);
}

// the cell's key as 32-bit words in the warp's shared memory (pushes copy it)
__device__ __forceinline__ void wload_key(WarpSh &S, const Arena &ar, int64_t cell)
{
    const int lane = threadIdx.x & 31;
    for (int w = lane; w < ar.kw; w += 32) {
        const unsigned long long x = __ldcg(ar.keys + cell * ar.kw + w);
        S.key[2 * w] = (unsigned)x;
        S.key[2 * w + 1] = (unsigned)(x >> 32);
    }
}

// The cell's rows view, key and face plane a_F in the warp's shared memory, then (lane 0) the
// face plane's FP32 frame and the square about the box section: the initial polygon in buffer 0
// (planes N + 6 .. N + 9).  Returns its vertex count, 0 when a_F has no normal.
__device__ int wcell_setup(const MarchArgs &a, WarpSh &S, int64_t cell, int N, WRows &rv)
{
    const int lane = threadIdx.x & 31;
    rv.p = reinterpret_cast<const float4 *>(a.rows_in) + (cell - a.begin) * 2 * (int64_t)(N + 1);
    rv.N = N;
    rv.box = a.box_hi;
    rv.box_lo = a.box_lo;
    rv.S = &S;
    wload_key(S, a.ar, cell);
    if (lane < 4) {
        const float h = reinterpret_cast<const float *>(rv.p + N)[lane];
        const float l = reinterpret_cast<const float *>(rv.p + 2 * N + 1)[lane];   // lo block: N + 1 + N
        S.aF[lane] = (double)h + (double)l;
        S.aFhi[lane] = h;
    }
    __syncwarp();
    int m = 0;
    if (lane == 0) {
        const float F[4] = {(float)S.aF[0], (float)S.aF[1], (float)S.aF[2], (float)S.aF[3]};
        const float nn = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
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
            const float d[4][3] = {{-w[0], -w[1], -w[2]}, {u[0], u[1], u[2]}, {w[0], w[1], w[2]}, {-u[0], -u[1], -u[2]}};
            const float cu[4] = {-1.0f, 1.0f, 1.0f, -1.0f}, cw[4] = {-1.0f, -1.0f, 1.0f, 1.0f};
            for (int i = 0; i < 4; ++i) {
                S.sq[i][0] = d[i][0]; S.sq[i][1] = d[i][1]; S.sq[i][2] = d[i][2];
                S.sq[i][3] = -(d[i][0] * p0[0] + d[i][1] * p0[1] + d[i][2] * p0[2]) - sz;
                for (int c = 0; c < 3; ++c) {
                    const float x = p0[c] + sz * (cu[i] * u[c] + cw[i] * w[c]);
                    S.pv[0][i][c] = (double)x;
                    S.pf[0][i][c] = x;
                }
                S.pe[0][i] = N + kBoxPlanes + i;
            }
            m = 4;
        }
    }
    m = __shfl_sync(0xffffffffu, m, 0);
    __syncwarp();
    return m;
}

// A close call of the FP32 test: row k at the FP64 vertex v6 from the exact pair, against the
// vertex's own error (|r|_1 dvb), the tolerance band and the FP64 evaluation's rounding.
// Returns 1 when the row is violated, 2 when the vertex is within the band (the FP64 path
// decides), 0 when it holds.  Out of line: the FP32 test decides nearly every pair.
__device__ __noinline__ int wclose(const WRows &rv, int k, const double *v6, float rl1, float dvb, float delta)
{
    double r6[4];
    rv.f64(k, r6);
    const float4 h = rv.hi(k);
    const float band = delta * sqrtf(h.x * h.x + h.y * h.y + h.z * h.z);   // delta |r|: the tolerance band
    const double s6 = r6[0] * v6[0] + r6[1] * v6[1] + r6[2] * v6[2] + r6[3];
    const double m6 = fabs(r6[0] * v6[0]) + fabs(r6[1] * v6[1]) + fabs(r6[2] * v6[2]) + fabs(r6[3]);
    const double B6 = (double)rl1 * 1.0001 * (double)dvb + (double)band + 1e-15 * m6;
    if (s6 > B6) return 1;
    return s6 >= -B6 ? 2 : 0;
}

// The certified all-row check of the polygon in buffer buf (FP64 vertices): every row at every
// vertex in FP32 with a bound, close calls in FP64 from the exact pair; violated rows are cut in
// (FP64) and the check repeats, at most kWMaxFix rounds.  Returns true when the cell must go to
// the block kernel (a row within the band, a violated row that is already an edge, too many
// violators or rounds, a cut that fails).
__device__ bool wcheck(const MarchArgs &a, WarpSh &S, const WRows &rv, int N, int &m, int &buf, int &rounds,
                       int &ncut, int &cell_close)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const int NC = N + kBoxPlanes;
    const float delta = (float)a.delta * 1.01f;
    bool fallback = false;
    while (true) {
        for (int i = lane; i < m; i += 32) {
            const double *v = S.pv[buf][i];
            const float x = (float)v[0], y = (float)v[1], z = (float)v[2];
            // the bound on the FP32 test of row r at this vertex (evaluation, the dropped lo words,
            // the vertex rounded to FP32: 8.5 u (|r|_1 |v|_inf + |r_3|); the FP64 vertex's own error:
            // |r|_1 dvb) is |r|_1 w + c_r with w = 8.5 u max(1, |v|_inf) + dvb and c_r = 8.5 u |r_3|
            // + delta |r| (|r . v| <= |r|_1 |v|_inf; each coordinate within half an ulp of v's)
            const float X = fmaxf(1.0f, fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z)))) * 1.0001f;
            S.vf[i] = make_float4(x, y, z, __fmaf_ru(8.5f * kWU, X, S.dvb[i]));
            S.ve[i] = make_int2(S.pe[buf][i == 0 ? m - 1 : i - 1], S.pe[buf][i]);
        }
        if (lane == 0) S.nviol = 0;
        __syncwarp();
        bool amb = false;
        int close = 0;
        for (int k0 = lane; k0 < NC; k0 += 32 * 4) {
            float4 rr[4];
            float rl1[4], cr[4];
            bool viol[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = k0 + 32 * u;
                rr[u] = k < N ? __ldg(rv.p + k) : (k < NC ? rv.hi(k) : make_float4(0.0f, 0.0f, 0.0f, 0.0f));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 r = rr[u];
                const float n2 = r.x * r.x + r.y * r.y + r.z * r.z;
                // a zero normal (a constant row, which holds in its own cell) or no row: skipped
                rl1[u] = n2 == 0.0f ? -1.0f : fabsf(r.x) + fabsf(r.y) + fabsf(r.z);
                cr[u] = __fmaf_ru(8.5f * kWU, fabsf(r.w), delta * sqrtf(n2));   // + delta |r|: the tolerance band
                viol[u] = false;
            }
            for (int i = 0; i < m; ++i) {
                const float4 V = S.vf[i];
                const int2 E = S.ve[i];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = k0 + 32 * u;
                    if (rl1[u] < 0.0f || k == E.x || k == E.y) continue;
                    const float4 r = rr[u];
                    const float sl = fmaf(r.x, V.x, fmaf(r.y, V.y, fmaf(r.z, V.z, r.w)));
                    const float B = __fmaf_ru(rl1[u], V.w, cr[u]);
                    if (sl > B) { viol[u] = true; continue; }
                    if (sl >= -B) {                        // close call: FP64 from the exact pair
                        ++close;
                        const int c = wclose(rv, k, S.pv[buf][i], rl1[u], S.dvb[i], delta);
                        viol[u] |= c == 1;
                        amb |= c == 2;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!viol[u]) continue;
                const int k = k0 + 32 * u;
                for (int i = 0; i < m; ++i) amb |= S.pe[buf][i] == k;   // a spurious FP32 cut
                const int p = atomicAdd(&S.nviol, 1);
                if (p < kWViol) S.viol[p] = k;
                else amb = true;
            }
        }
        for (int o = 16; o > 0; o >>= 1) close += __shfl_xor_sync(FULL, close, o);
        cell_close += close;
        if (__any_sync(FULL, amb)) { fallback = true; break; }
        __syncwarp();
        const int nviol = S.nviol;
        if (nviol == 0) break;
        if (rounds + 1 >= kWMaxFix) { fallback = true; break; }
        for (int t = 0; t < nviol && m > 0; ++t) {
            bool sw;
            const int nm = wcut<double>(S, S.pv, m, buf, S.viol[t], 0.0, S.aF, rv, &sw);
            if (nm < 0) { fallback = true; break; }
            if (sw) buf ^= 1;
            m = nm;
        }
        ncut += nviol;
        if (fallback || m == 0) { fallback = true; break; }
        if (!wfinal(S, m, buf, rv)) { fallback = true; break; }
        ++rounds;
    }
    return fallback;
}

// a6 emit, a7 march for a solved cell: the face record (empty when it has fewer than 3 vertices,
// a square edge, or no area), then one push per neuron edge; returns whether a face was written
__device__ bool wemit(const MarchArgs &a, WarpSh &S, int64_t cell, int net_id, int N, int m, int buf)
{
    const int lane = threadIdx.x & 31;
    const Arena &ar = a.ar;
    int emit = m >= 3 ? m : 0;
    for (int i = 0; i < m; ++i)
        if (S.pe[buf][i] >= N + kBoxPlanes) emit = 0;     // a square edge: the plane misses the box
    if (emit) {
        const double *p0 = S.pv[buf][0];
        double nx = 0.0, ny = 0.0, nz = 0.0;
        for (int i = lane + 1; i < m - 1; i += 32) {
            const double *p = S.pv[buf][i], *q = S.pv[buf][i + 1];
            const double ax = p[0] - p0[0], ay = p[1] - p0[1], az = p[2] - p0[2];
            const double bx = q[0] - p0[0], by = q[1] - p0[1], bz = q[2] - p0[2];
            nx += ay * bz - az * by; ny += az * bx - ax * bz; nz += ax * by - ay * bx;
        }
        nx = warp_sum(nx); ny = warp_sum(ny); nz = warp_sum(nz);
        const double amin = 2e-24 * a.box * a.box;    // twice the smallest kept area
        if (!(nx * nx + ny * ny + nz * nz > amin * amin)) emit = 0;
    }
    if (emit > ar.maxv) {
        if (lane == 0) atomicOr(ar.counters + kStatus, kStFaceVerts);
        emit = 0;
    }
    if (lane == 0) ar.nverts[cell] = emit;
    if (emit) {
        for (int i = lane; i < m; i += 32) {
            ar.edges[cell * ar.maxv + i] = S.pe[buf][i];
            double *v = ar.verts + (cell * ar.maxv + i) * 3;
            v[0] = S.pv[buf][i][0]; v[1] = S.pv[buf][i][1]; v[2] = S.pv[buf][i][2];
        }
        const unsigned long long h = __ldcg(ar.hash + cell);
        // the entry point of each neighbour (the midpoint of the shared edge), one edge per lane,
        // kept in the FP32 polygon's buffer (buf ^ 1 is free: the face is in buf)
        float (*mid)[3] = S.pf[buf ^ 1];
        for (int i = lane; i < m; i += 32) {
            const double *p = S.pv[buf][i], *q = S.pv[buf][i + 1 == m ? 0 : i + 1];
            mid[i][0] = (float)(0.5 * (p[0] + q[0]));
            mid[i][1] = (float)(0.5 * (p[1] + q[1]));
            mid[i][2] = (float)(0.5 * (p[2] + q[2]));
        }
        __syncwarp();
        for (int i = 0; i < m; ++i) {
            const int e = S.pe[buf][i];
            if (e >= N) continue;
            insert_neighbor_warp(ar, S.key, cell, net_id, (unsigned)e, h ^ ar.zob[e], mid[i][0], mid[i][1], mid[i][2],
                                 false);
        }
    }
    return emit != 0;
}

}  // namespace

int clip_warp_smem_bytes() { return warp_smem_bytes(); }

#ifndef AM_CLIP_MIN_BLOCKS
#define AM_CLIP_MIN_BLOCKS 3
#endif
__global__ void __launch_bounds__(kWW * 32, AM_CLIP_MIN_BLOCKS) clip_warp_kernel(MarchArgs a)
{
    extern __shared__ __align__(16) unsigned char wsm[];
    WarpSh &S = reinterpret_cast<WarpSh *>(wsm)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const Arena &ar = a.ar;
    unsigned long long n_solved = 0, n_empty = 0, n_fix = 0, n_cuts = 0, n_close = 0, n_fb = 0;
    const int64_t stride = (int64_t)gridDim.x * kWW;
    // with a.work the warps take cells one at a time from a shared counter (cells differ in
    // their cost: the cuts, the fix-up rounds), else in a fixed stride
    auto next = [&](int64_t cur) -> int64_t {
        if (!a.work) return cur + stride;
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.work, 1ull);
        return a.begin + (int64_t)__shfl_sync(FULL, t, 0);
    };
    for (int64_t cell = a.work ? next(0) : a.begin + (int64_t)blockIdx.x * kWW + (threadIdx.x >> 5); cell < a.end;
         cell = next(cell)) {
        if (__ldcg(ar.nverts + cell) == -2) continue;          // a duplicate seed id: never solved
        const int net_id = __ldcg(ar.net + cell);
        const int N = a.nets[net_id].N;
        WRows rv;
        int m = wcell_setup(a, S, cell, N, rv);
        bool fallback = m == 0;
        // ---- candidates: per lane the two best of the rows it scans
        const float px = __ldcg(ar.entry_pt + cell * 3), py = __ldcg(ar.entry_pt + cell * 3 + 1),
                    pz = __ldcg(ar.entry_pt + cell * 3 + 2);
        const int entry = __ldcg(ar.entry_plane + cell);
        const bool learned = a.candidates == kCandLearned && a.scores_in && a.prop.n_out == N;
        const __nv_bfloat16 *sc = learned ? a.scores_in + (cell - a.begin) * (int64_t)a.scores_ld : nullptr;
        float b1 = 3.0e38f, b2 = 3.0e38f, b3 = 3.0e38f, s3 = 3.0e38f;
        int k1 = -1, k2 = -1, k3 = -1;
        if (!fallback) {
            auto consider = [&](int k, const float4 r, float score) {
                const float n2 = r.x * r.x + r.y * r.y + r.z * r.z;
                if (n2 == 0.0f) return;
                const float d = fabsf(r.x * px + r.y * py + r.z * pz + r.w) * rsqrtf(n2);
                if (d < b1) { b2 = b1; k2 = k1; b1 = d; k1 = k; }
                else if (d < b2) { b2 = d; k2 = k; }
                if (learned && k < N) {
                    // the learned proposal adds the row it scores highest among this lane's
                    const float q = k == entry ? -3.0e37f : -score;
                    if (q < s3) { s3 = q; k3 = k; b3 = d; }
                }
            };
            // the neuron rows and their scores, 8 of each in flight per lane; then the box rows
            // (lanes 0..5)
            for (int k0 = lane; k0 < N; k0 += 32 * 8) {
                float4 r[8];
                float q[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = k0 + 32 * u;
                    r[u] = k < N ? __ldg(rv.p + k) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    q[u] = learned && k < N ? __bfloat162float(sc[k]) : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (k0 + 32 * u < N) consider(k0 + 32 * u, r[u], q[u]);
            }
            if (lane < kBoxPlanes) consider(N + lane, rv.hi(N + lane), 0.0f);
            if (k3 == k1 || k3 == k2) k3 = -1;            // already a candidate
        }
        // ---- the candidate clip (FP32): nearest cutting row first; a row that holds on the
        //      polygon holds on every later (smaller) one and retires
        int buf = 0, ncut = 0;
        {
            // up to three candidate slots per lane, cut nearest first (the learned slot too)
            const int kk[3] = {k1, k2, k3};
            const unsigned key[3] = {order_key(b1), order_key(b2), order_key(b3)};
            bool live[3] = {k1 >= 0, k2 >= 0, k3 >= 0};
            float cr[3][4], cri[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (kk[j] >= 0) rv.f32(kk[j], cr[j]);
                else cr[j][0] = cr[j][1] = cr[j][2] = cr[j][3] = 0.0f;
                cri[j] = kk[j] >= 0 ? rsqrtf(cr[j][0] * cr[j][0] + cr[j][1] * cr[j][1] + cr[j][2] * cr[j][2]) : 0.0f;
            }
            while (!fallback && m > 0) {
                bool c[3] = {false, false, false};
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (!live[j]) continue;
                    for (int i = 0; i < m && !c[j]; ++i) c[j] = wpdist(cr[j], cri[j], S.pf[buf][i]) > 1e-7f;
                }
#pragma unroll
                for (int j = 0; j < 3; ++j) live[j] = c[j];
                if (!__any_sync(FULL, c[0] || c[1] || c[2])) break;
                unsigned mine = 0xffffffffu;
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (c[j]) mine = min(mine, key[j]);
                const unsigned kmin = __reduce_min_sync(FULL, mine);
                unsigned cand = 0xffffffffu;
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (c[j] && key[j] == kmin) cand = min(cand, (unsigned)kk[j]);
                const int kc = (int)__reduce_min_sync(FULL, cand);
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (kk[j] == kc) live[j] = false;
                bool sw;
                const int nm = wcut<float>(S, S.pf, m, buf, kc, 1e-7f, S.aFhi, rv, &sw);
                if (nm < 0) { fallback = true; break; }
                if (sw) buf ^= 1;
                m = nm;
                ++ncut;
            }
        }
        // an FP32 pass that emptied the polygon proves nothing: the FP64 fallback decides
        if (m == 0) fallback = true;
        if (!fallback) fallback = !wfinal(S, m, buf, rv);
        if (!fallback && a.chk && m <= kChkMaxV) {
            // the dense check runs on the tensor cores (check_tc); the finish pass emits the cell
            unsigned long long p = 0;
            if (lane == 0) p = atomicAdd(a.chk_count, 1ull);
            p = __shfl_sync(FULL, p, 0);
            CheckRec &R = a.chk[p];
            if (lane == 0) { R.cell = (int32_t)cell; R.m = m; }
            for (int i = lane; i < m; i += 32) {
                R.pe[i] = S.pe[buf][i];
                R.v[i][0] = S.pv[buf][i][0]; R.v[i][1] = S.pv[buf][i][1]; R.v[i][2] = S.pv[buf][i][2];
            }
            n_cuts += (unsigned long long)ncut;
            __syncwarp();
            continue;
        }
        // ---- the all-row check, certified; violators are cut in (FP64) and the check repeats
        int rounds = 0, cell_close = 0;
        if (!fallback) fallback = wcheck(a, S, rv, N, m, buf, rounds, ncut, cell_close);
        if (fallback) {
            // the block kernel solves this cell (double-float, then FP64 where needed)
            if (lane == 0) {
                const unsigned long long p = atomicAdd(a.fb_count, 1ull);
                a.fb_list[p] = (int32_t)cell;
            }
            n_fb += 1;
            continue;
        }
        // ---- a6 emit, a7 march
        const bool emitted = wemit(a, S, cell, net_id, N, m, buf);
        n_solved += 1;
        if (!emitted) n_empty += 1;
        if (rounds) n_fix += 1;
        n_cuts += (unsigned long long)ncut;
        n_close += (unsigned long long)cell_close;
        __syncwarp();
    }
    if (lane == 0) {
        unsigned long long *C = ar.counters;
        if (n_solved) atomicAdd(C + kSolved, n_solved);
        if (n_empty) atomicAdd(C + kEmpty, n_empty);
        if (n_fix) atomicAdd(C + kFixups, n_fix);
        if (n_cuts) atomicAdd(C + kCuts, n_cuts);
        if (n_close) atomicAdd(C + kCloseCalls, n_close);
        if (n_fb) atomicAdd(C + kWarpFallback, n_fb);
    }
}

// After check_tc: one warp per record.  A cell whose rows all hold is emitted and pushes its
// neighbours; a cell with a violated or undecided row gets the warp's own check (violators cut in,
// FP64 close calls), and what that cannot decide goes to the block kernel's list.
__global__ void __launch_bounds__(kWW * 32) clip_warp_finish_kernel(MarchArgs a)
{
    extern __shared__ __align__(16) unsigned char wsm[];
    WarpSh &S = reinterpret_cast<WarpSh *>(wsm)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const Arena &ar = a.ar;
    unsigned long long n_solved = 0, n_empty = 0, n_fix = 0, n_cuts = 0, n_close = 0, n_fb = 0;
    const int64_t n = (int64_t)__ldcg(a.chk_count);
    const int64_t stride = (int64_t)gridDim.x * kWW;
    for (int64_t idx = (int64_t)blockIdx.x * kWW + (threadIdx.x >> 5); idx < n; idx += stride) {
        const CheckRec &R = a.chk[idx];
        const int64_t cell = R.cell;
        int m = R.m, buf = 0, rounds = 0, ncut = 0, cell_close = 0;
        const int net_id = __ldcg(ar.net + cell);
        const int N = a.nets[net_id].N;
        bool fallback = false;
        if (a.chk_status[idx] == 0) {
            wload_key(S, ar, cell);
        } else {
            WRows rv;
            fallback = wcell_setup(a, S, cell, N, rv) == 0;   // key, a_F and the square's rows
            for (int i = lane; i < m; i += 32) {
                S.pe[0][i] = R.pe[i];
            }
            __syncwarp();
            if (!fallback) fallback = !wfinal(S, m, 0, rv);     // the same FP64 vertices and their bounds
            if (!fallback) fallback = wcheck(a, S, rv, N, m, buf, rounds, ncut, cell_close);
        }
        if (fallback) {
            if (lane == 0) {
                const unsigned long long p = atomicAdd(a.fb_count, 1ull);
                a.fb_list[p] = (int32_t)cell;
            }
            n_fb += 1;
            continue;
        }
        if (a.chk_status[idx] == 0) {
            for (int i = lane; i < m; i += 32) {
                S.pe[0][i] = R.pe[i];
                S.pv[0][i][0] = R.v[i][0]; S.pv[0][i][1] = R.v[i][1]; S.pv[0][i][2] = R.v[i][2];
            }
        }
        __syncwarp();
        const bool emitted = wemit(a, S, cell, net_id, N, m, buf);
        n_solved += 1;
        if (!emitted) n_empty += 1;
        if (rounds) n_fix += 1;
        n_cuts += (unsigned long long)ncut;
        n_close += (unsigned long long)cell_close;
        __syncwarp();
    }
    if (lane == 0) {
        unsigned long long *C = ar.counters;
        if (n_solved) atomicAdd(C + kSolved, n_solved);
        if (n_empty) atomicAdd(C + kEmpty, n_empty);
        if (n_fix) atomicAdd(C + kFixups, n_fix);
        if (n_cuts) atomicAdd(C + kCuts, n_cuts);
        if (n_close) atomicAdd(C + kCloseCalls, n_close);
        if (n_fb) atomicAdd(C + kWarpFallback, n_fb);
    }
}

static int g_clip_resident = 0;       // clip_warp_kernel blocks resident on the whole GPU at once

cudaError_t prepare_clip_warp()
{
    cudaError_t e = cudaFuncSetAttribute(clip_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, warp_smem_bytes());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(clip_warp_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, warp_smem_bytes());
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, clip_warp_kernel, kWW * 32, warp_smem_bytes());
    if (e != cudaSuccess) return e;
    g_clip_resident = std::max(1, sms * per_sm);
    return cudaSuccess;
}

void launch_clip_warp(const MarchArgs &a, cudaStream_t st)
{
    const int64_t n = a.end - a.begin;
    // with a work counter: one resident wave that drains the cells; else one warp per cell
    const int64_t cap = a.work && g_clip_resident > 0 ? g_clip_resident : 152 * 64;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + kWW - 1) / kWW, cap));
    clip_warp_kernel<<<grid, kWW * 32, warp_smem_bytes(), st>>>(a);
}

void launch_clip_warp_finish(const MarchArgs &a, cudaStream_t st)
{
    const int64_t n = a.end - a.begin;                 // the records are at most the cells
    const int grid = (int)std::min<int64_t>((n + kWW - 1) / kWW, 152 * 16);
    clip_warp_finish_kernel<<<grid, kWW * 32, warp_smem_bytes(), st>>>(a);
}

}  // namespace am
