/*
 * am_oracle.c -- plain FP64 CPU oracle for analytic marching
 * (Lei, Jia & Ma, "Analytic Marching: an analytic meshing solution from deep
 *  implicit surface networks", arXiv 2106.10031).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file; the library's product path
 * never does.  It shares no code, header or table with the CUDA path.
 *
 * Everything here is deliberately literal and slow: loops, no BLAS, no
 * blocking, FP64 throughout.  Affine maps are carried in homogeneous form, a
 * row [a_x a_y a_z | a_0] acting on [x; 1]: this is how the biases, which the
 * paper leaves out of its notation (Sec. 2.2), enter every formula.
 *
 * Network format (packed by oracle/oracle.py):
 *   desc  = [L, in_dim, skip_layer, n_1, ..., n_L]          (int32)
 *   param = W_1, b_1, ..., W_L, b_L, w_out, b_out, z        (float64)
 *     W_l is n_l x fan_l row-major; fan_1 = in_dim;
 *     fan_l = n_{l-1} (+ in_dim when l == skip_layer);
 *     z (in_dim - 3 values) is the fixed latent code: the net's input is [x; z].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_LAYERS 64

typedef struct {
    int L, in_dim, skip, N;
    int n[ORC_MAX_LAYERS + 1];     /* n[1..L] */
    int fan[ORC_MAX_LAYERS + 1];
    const double *W[ORC_MAX_LAYERS + 1], *b[ORC_MAX_LAYERS + 1];
    const double *w_out, *z;
    double b_out;
} orc_net;

static int orc_parse(const int *desc, const double *prm, orc_net *net)
{
    int l;
    const double *p = prm;
    net->L = desc[0];
    net->in_dim = desc[1];
    net->skip = desc[2];
    if (net->L < 1 || net->L > ORC_MAX_LAYERS || net->in_dim < 3) return -1;
    net->N = 0;
    for (l = 1; l <= net->L; ++l) {
        net->n[l] = desc[2 + l];
        if (net->n[l] < 1) return -1;
        net->N += net->n[l];
    }
    for (l = 1; l <= net->L; ++l) {
        net->fan[l] = (l == 1) ? net->in_dim : net->n[l - 1] + (l == net->skip ? net->in_dim : 0);
        net->W[l] = p; p += (size_t)net->n[l] * net->fan[l];
        net->b[l] = p; p += net->n[l];
    }
    net->w_out = p; p += net->n[net->L];
    net->b_out = *p; p += 1;
    net->z = p;
    return 0;
}

int orc_num_neurons(const int *desc)
{
    int l, N = 0;
    for (l = 1; l <= desc[0]; ++l) N += desc[2 + l];
    return N;
}

/* ------------------------------------------------------------------------------------------
 * Forward pass (Sec. 2.2, Eq. 1 with biases): the pre-activations a_lk(x) of every hidden
 * neuron, in layer order, and F(x) = w_out . h_L + b_out.
 */
int orc_forward(const int *desc, const double *prm, const double *x, double *pre, double *F)
{
    orc_net net;
    double *u0, *h, *in, *hn;
    int l, k, j, row0 = 0, fan_max = 0;
    if (orc_parse(desc, prm, &net)) return -1;
    for (l = 1; l <= net.L; ++l) {
        if (net.fan[l] > fan_max) fan_max = net.fan[l];
        if (net.n[l] > fan_max) fan_max = net.n[l];
    }
    u0 = (double *)malloc(sizeof(double) * net.in_dim);
    in = (double *)malloc(sizeof(double) * fan_max);
    h = (double *)malloc(sizeof(double) * fan_max);
    hn = (double *)malloc(sizeof(double) * fan_max);
    for (j = 0; j < 3; ++j) u0[j] = x[j];
    for (j = 3; j < net.in_dim; ++j) u0[j] = net.z[j - 3];
    for (l = 1; l <= net.L; ++l) {
        int fan = net.fan[l];
        if (l == 1) {
            memcpy(in, u0, sizeof(double) * net.in_dim);
        } else {
            memcpy(in, h, sizeof(double) * net.n[l - 1]);
            if (l == net.skip) memcpy(in + net.n[l - 1], u0, sizeof(double) * net.in_dim);
        }
        for (k = 0; k < net.n[l]; ++k) {
            double a = net.b[l][k];
            for (j = 0; j < fan; ++j) a += net.W[l][(size_t)k * fan + j] * in[j];
            if (pre) pre[row0 + k] = a;
            hn[k] = a > 0.0 ? a : 0.0;              /* g = ReLU */
        }
        memcpy(h, hn, sizeof(double) * net.n[l]);
        row0 += net.n[l];
    }
    if (F) {
        double f = net.b_out;
        for (k = 0; k < net.n[net.L]; ++k) f += net.w_out[k] * h[k];
        *F = f;
    }
    free(u0); free(in); free(h); free(hn);
    return 0;
}

/* State functional, Def. 2 (Eq. 2-4): s_lk = 1 iff a_lk(x) > 0 (a tie gives 0). */
int orc_state(const int *desc, const double *prm, const double *x, unsigned char *s, double *F)
{
    int k, N = orc_num_neurons(desc);
    double *pre = (double *)malloc(sizeof(double) * N);
    int rc = orc_forward(desc, prm, x, pre, F);
    for (k = 0; rc == 0 && k < N; ++k) s[k] = pre[k] > 0.0 ? 1 : 0;
    free(pre);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * Region-wise affine maps, Lemma 1 and Cor. 1 (Eqs. 6-9), in homogeneous form.
 *   In_l : map from [x;1] to the input of hidden layer l   (fan_l x 4)
 *   Z_l  = W_l In_l + b_l e_4^T                              (n_l x 4): rows a^r_lk
 *   H_l  = diag(s_l) Z_l  (= W^r_l applied to In_l)
 *   a_F  = w_out^T H_L + b_out e_4^T
 * In_1 maps [x;1] to [x; z]; In_l = H_{l-1}, stacked over In_1 at the skip layer.
 * Output A is N x 4 (layer order), aF is 4.
 */
int orc_compose(const int *desc, const double *prm, const unsigned char *s, double *A, double *aF)
{
    orc_net net;
    double *X0, *In, *H, *Z;
    int l, k, j, c, row0 = 0, fan_max = 0;
    if (orc_parse(desc, prm, &net)) return -1;
    for (l = 1; l <= net.L; ++l) {
        if (net.fan[l] > fan_max) fan_max = net.fan[l];
        if (net.n[l] > fan_max) fan_max = net.n[l];
    }
    X0 = (double *)calloc((size_t)net.in_dim * 4, sizeof(double));
    In = (double *)calloc((size_t)fan_max * 4, sizeof(double));
    H = (double *)calloc((size_t)fan_max * 4, sizeof(double));
    Z = (double *)calloc((size_t)fan_max * 4, sizeof(double));
    for (j = 0; j < 3; ++j) X0[j * 4 + j] = 1.0;
    for (j = 3; j < net.in_dim; ++j) X0[j * 4 + 3] = net.z[j - 3];
    for (l = 1; l <= net.L; ++l) {
        int fan = net.fan[l];
        if (l == 1) {
            memcpy(In, X0, sizeof(double) * 4 * net.in_dim);
        } else {
            memcpy(In, H, sizeof(double) * 4 * net.n[l - 1]);
            if (l == net.skip) memcpy(In + 4 * net.n[l - 1], X0, sizeof(double) * 4 * net.in_dim);
        }
        for (k = 0; k < net.n[l]; ++k) {
            for (c = 0; c < 4; ++c) {
                double acc = 0.0;
                for (j = 0; j < fan; ++j) acc += net.W[l][(size_t)k * fan + j] * In[j * 4 + c];
                Z[k * 4 + c] = acc + (c == 3 ? net.b[l][k] : 0.0);
            }
            for (c = 0; c < 4; ++c) {
                A[(size_t)(row0 + k) * 4 + c] = Z[k * 4 + c];
                H[k * 4 + c] = s[row0 + k] ? Z[k * 4 + c] : 0.0;
            }
        }
        row0 += net.n[l];
    }
    for (c = 0; c < 4; ++c) {
        double acc = 0.0;
        for (k = 0; k < net.n[net.L]; ++k) acc += net.w_out[k] * H[k * 4 + c];
        aF[c] = acc + (c == 3 ? net.b_out : 0.0);
    }
    free(X0); free(In); free(H); free(Z);
    return 0;
}

/* Analytic cell system (Eq. 10): rows (1 - 2 s_k) a_k, followed by the six box rows
 * [+-e_i | -B] with ids N..N+5 in the order +x, -x, +y, -y, +z, -z.  C is (N+6) x 4. */
int orc_cell_rows(const int *desc, const double *prm, const unsigned char *s, double B,
                  double *C, double *aF)
{
    int k, c, i, N = orc_num_neurons(desc);
    int rc = orc_compose(desc, prm, s, C, aF);
    if (rc) return rc;
    for (k = 0; k < N; ++k) {
        double sg = 1.0 - 2.0 * (double)s[k];
        for (c = 0; c < 4; ++c) C[(size_t)k * 4 + c] *= sg;
    }
    for (i = 0; i < 6; ++i) {
        double *r = C + (size_t)(N + i) * 4;
        r[0] = r[1] = r[2] = 0.0;
        r[i / 2] = (i % 2 == 0) ? 1.0 : -1.0;
        r[3] = -B;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Vertex equation system (Eq. 11) with biases: [c_t; c_u; a_F] [v; 1] = 0, i.e. a 3x3 solve
 * for v, by Gaussian elimination with partial pivoting.  Returns -1 when singular.
 */
static int orc_solve3(const double *r0, const double *r1, const double *r2, double *v)
{
    double M[3][4];
    const double *r[3];
    int i, j, k, p;
    r[0] = r0; r[1] = r1; r[2] = r2;
    for (i = 0; i < 3; ++i) {
        for (j = 0; j < 3; ++j) M[i][j] = r[i][j];
        M[i][3] = -r[i][3];
    }
    for (k = 0; k < 3; ++k) {
        p = k;
        for (i = k + 1; i < 3; ++i) if (fabs(M[i][k]) > fabs(M[p][k])) p = i;
        if (M[p][k] == 0.0) return -1;
        if (p != k) for (j = 0; j < 4; ++j) { double t = M[k][j]; M[k][j] = M[p][j]; M[p][j] = t; }
        for (i = k + 1; i < 3; ++i) {
            double f = M[i][k] / M[k][k];
            for (j = k; j < 4; ++j) M[i][j] -= f * M[k][j];
        }
    }
    for (i = 2; i >= 0; --i) {
        double acc = M[i][3];
        for (j = i + 1; j < 3; ++j) acc -= M[i][j] * v[j];
        v[i] = acc / M[i][i];
    }
    for (i = 0; i < 3; ++i) if (!isfinite(v[i])) return -1;
    return 0;
}

static double orc_norm3(const double *r) { return sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]); }

/* Signed Euclidean distance of v from the plane of row r (positive = violated). */
static double orc_dist(const double *r, const double *v)
{
    return (r[0] * v[0] + r[1] * v[1] + r[2] * v[2] + r[3]) / orc_norm3(r);
}

/* Validity of a candidate vertex (Alg. 1 step 8 / Alg. 2): every row of the cell system
 * other than the two defining ones holds, up to the distance tolerance delta.  Rows with a
 * zero normal hold iff their constant is <= 0.  *ndeg counts rows within delta. */
static int orc_valid(int M, const double *C, const double *v, int t, int u, double delta, int *ndeg)
{
    int k, nd = 0;
    for (k = 0; k < M; ++k) {
        const double *r = C + (size_t)k * 4;
        double d;
        if (k == t || k == u) continue;
        if (orc_norm3(r) == 0.0) {
            if (r[3] > 0.0) return 0;
            continue;
        }
        d = orc_dist(r, v);
        if (d > delta) return 0;
        if (d >= -delta) ++nd;
    }
    if (ndeg) *ndeg = nd;
    return 1;
}

typedef struct { double d; int k; } orc_key;

static int orc_cmp(const void *a, const void *b)
{
    const orc_key *x = (const orc_key *)a, *y = (const orc_key *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return x->k - y->k;
}

/* ------------------------------------------------------------------------------------------
 * Pivoting enumeration, Alg. 2 (Sec. 4.2.1, App. B).
 *   M rows C (cell system incl. box rows), face plane aF, a true boundary `start` (H*) and a
 *   point x on the face.  Planes are ordered by their Euclidean distance to x.  The first
 *   loop finds a vertex on H*; the second walks from plane to plane (excluding the current
 *   and the previous one), each time taking the first valid candidate in the sorted order,
 *   until the walk comes back to H*.
 * Outputs, in walk order: vertices V (nv x 3) and, for vertex i, the two planes whose
 * intersection (with the face plane) it is: pairs[2i] (the plane walked along before it)
 * and pairs[2i+1] (the plane walked along after it).  *ndeg sums, over accepted vertices,
 * the rows other than the defining pair that lie within delta of the vertex.
 * Returns 0, or -1 (bad input), -2 (no vertex on H*), -3 (walk did not close).
 */
int orc_pivot(int M, const double *C, const double *aF, int start, const double *x, double delta,
              int max_v, double *V, int *pairs, int *nv_out, int *ndeg_out)
{
    orc_key *ord;
    int m = 0, i, nv = 0, nd, ndeg = 0, t, tprev, found, steps, rc = 0;
    double v[3];
    if (start < 0 || start >= M || max_v < 3) return -1;
    ord = (orc_key *)malloc(sizeof(orc_key) * M);
    for (i = 0; i < M; ++i) {
        const double *r = C + (size_t)i * 4;
        double nr = orc_norm3(r);
        if (nr == 0.0) continue;
        ord[m].d = fabs(r[0] * x[0] + r[1] * x[1] + r[2] * x[2] + r[3]) / nr;
        ord[m].k = i;
        ++m;
    }
    qsort(ord, m, sizeof(orc_key), orc_cmp);

    /* first loop: a valid vertex on H* */
    t = start; tprev = -1; found = 0;
    for (i = 0; i < m; ++i) {
        int u = ord[i].k;
        if (u == t) continue;
        if (orc_solve3(C + (size_t)t * 4, C + (size_t)u * 4, aF, v)) continue;
        if (!orc_valid(M, C, v, t, u, delta, &nd)) continue;
        V[0] = v[0]; V[1] = v[1]; V[2] = v[2];
        pairs[0] = t; pairs[1] = u;
        ndeg += nd; nv = 1;
        tprev = t; t = u; found = 1;
        break;
    }
    if (!found) { rc = -2; goto done; }

    /* second loop: walk around the face until the walk reaches H* again */
    for (steps = 0;; ++steps) {
        if (steps > M + 1 || nv >= max_v) { rc = -3; goto done; }
        found = 0;
        for (i = 0; i < m; ++i) {
            int u = ord[i].k;
            if (u == t || u == tprev) continue;
            if (orc_solve3(C + (size_t)t * 4, C + (size_t)u * 4, aF, v)) continue;
            if (!orc_valid(M, C, v, t, u, delta, &nd)) continue;
            V[3 * nv] = v[0]; V[3 * nv + 1] = v[1]; V[3 * nv + 2] = v[2];
            pairs[2 * nv] = t; pairs[2 * nv + 1] = u;
            ndeg += nd; ++nv;
            found = 1;
            if (u == start) goto done;
            tprev = t; t = u;
            break;
        }
        if (!found) { rc = -3; goto done; }
    }
done:
    free(ord);
    *nv_out = nv;
    if (ndeg_out) *ndeg_out = ndeg;
    return rc;
}

/* The row whose line on the face plane is nearest (in-plane distance) to the point x of the
 * face: |c.x + c_0| / |c - (c.n / n.n) n| with n the face normal.  For an interior point
 * that line carries an edge of the face, so it is a true boundary H* for Alg. 2.  Rows
 * parallel to the face plane are skipped.  Returns the row index, or -1. */
int orc_nearest_line(int M, const double *C, const double *aF, const double *x)
{
    int k, best = -1;
    double bd = INFINITY, nn = aF[0] * aF[0] + aF[1] * aF[1] + aF[2] * aF[2];
    if (nn == 0.0) return -1;
    for (k = 0; k < M; ++k) {
        const double *r = C + (size_t)k * 4;
        double cn = (r[0] * aF[0] + r[1] * aF[1] + r[2] * aF[2]) / nn, p[3], pn, d;
        p[0] = r[0] - cn * aF[0]; p[1] = r[1] - cn * aF[1]; p[2] = r[2] - cn * aF[2];
        pn = orc_norm3(p);
        if (pn == 0.0) continue;
        d = fabs(r[0] * x[0] + r[1] * x[1] + r[2] * x[2] + r[3]) / pn;
        if (d < bd) { bd = d; best = k; }
    }
    return best;
}

/* ------------------------------------------------------------------------------------------
 * Trigger by dichotomy along a ray (Sec. 4.3.2): bisect t in [0, R] on x(t) = o + t d,
 * keeping F(lo) and F(hi) of opposite sign, until both ends have the same state (one affine
 * cell) or max_halvings is reached.  Inside that cell F is affine along the segment, so the
 * root is t* = t_lo + F_lo / (F_lo - F_hi) (t_hi - t_lo).  Outputs the root, its cell state
 * and the number of halvings.  Returns 0, -1 (bad input), -4 (no sign change), -5 (no
 * common cell after max_halvings).
 */
int orc_seed_ray(const int *desc, const double *prm, const double *o, const double *d, double R,
                 int max_halvings, double *x_out, unsigned char *s_out, int *halvings)
{
    int N = orc_num_neurons(desc), it = 0, i, same = 0, rc = 0;
    unsigned char *slo = (unsigned char *)malloc(N), *shi = (unsigned char *)malloc(N);
    double tlo = 0.0, thi = R, flo, fhi, fm, xl[3], xh[3], xm[3];
    for (i = 0; i < 3; ++i) { xl[i] = o[i]; xh[i] = o[i] + R * d[i]; }
    if (orc_state(desc, prm, xl, slo, &flo) || orc_state(desc, prm, xh, shi, &fhi)) { rc = -1; goto out; }
    if (!(flo < 0.0 && fhi > 0.0) && !(flo > 0.0 && fhi < 0.0)) { rc = -4; goto out; }
    for (;;) {
        same = memcmp(slo, shi, N) == 0;
        if (same || it >= max_halvings) break;
        {
            double tm = 0.5 * (tlo + thi);
            for (i = 0; i < 3; ++i) xm[i] = o[i] + tm * d[i];
            if (orc_state(desc, prm, xm, s_out, &fm)) { rc = -1; goto out; }
            if ((fm < 0.0) == (flo < 0.0) && fm != 0.0) {
                tlo = tm; flo = fm; memcpy(slo, s_out, N);
            } else {
                thi = tm; fhi = fm; memcpy(shi, s_out, N);
            }
        }
        ++it;
    }
    if (!same) { rc = -5; goto out; }
    {
        double ts = tlo + flo / (flo - fhi) * (thi - tlo);
        for (i = 0; i < 3; ++i) x_out[i] = o[i] + ts * d[i];
        memcpy(s_out, slo, N);
    }
out:
    if (halvings) *halvings = it;
    free(slo); free(shi);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * Trigger by sphere tracing for an SDF (Sec. 4.3.1): from x_0, step
 *     x_{t+1} = x_t - eta F(x_t) grad F(x_t)
 * where grad F(x_t) is the gradient of the affine piece of the cell x_t lies in, i.e. the
 * first three entries of a_F composed (Cor. 1) for the state of x_t (a tie gives state 0).
 * The walk stops after max_steps steps, or earlier once |F(x_t)| <= eps.  Outputs the last
 * point, F there and the gradient of its cell, and the number of steps taken.  Returns 0,
 * -1 (bad input) or -6 (a cell with a zero gradient: the walk cannot move).
 */
int orc_sphere_trace(const int *desc, const double *prm, const double *x0, double eta, int max_steps,
                     double eps, double *x_out, double *F_out, double *g_out, int *steps)
{
    int N = orc_num_neurons(desc), t = 0, i, rc = 0;
    unsigned char *s = (unsigned char *)malloc(N);
    double *A = (double *)malloc(sizeof(double) * 4 * N);
    double x[3], F = 0.0, aF[4];
    if (!s || !A || max_steps < 0) { rc = -1; goto out; }
    for (i = 0; i < 3; ++i) x[i] = x0[i];
    for (;;) {
        if (orc_state(desc, prm, x, s, &F) || orc_compose(desc, prm, s, A, aF)) { rc = -1; goto out; }
        if (fabs(F) <= eps || t >= max_steps) break;
        if (aF[0] == 0.0 && aF[1] == 0.0 && aF[2] == 0.0) { rc = -6; break; }
        for (i = 0; i < 3; ++i) x[i] = x[i] - eta * F * aF[i];
        ++t;
    }
    for (i = 0; i < 3; ++i) { x_out[i] = x[i]; g_out[i] = aF[i]; }
    *F_out = F;
out:
    if (steps) *steps = t;
    free(s); free(A);
    return rc;
}
