/*
 * analytic_marching.h -- C ABI of the GB300 analytic-marching library.
 *
 * Analytic marching (Lei, Jia & Ma, arXiv 2106.10031) extracts the exact polygon mesh of
 * the zero level set of a ReLU MLP F = f o T (Sec. 2, Sec. 3).  Every linear region
 * (cell) of the MLP is labelled by its activation pattern s (Def. 2); inside a cell F is
 * affine (Lemma 1, Cor. 1), the cell is the polyhedron of Eq. 10 and its face is the
 * polygon of Eq. 12.  Algorithm 1 walks from cell to cell across the edges of the faces,
 * flipping the state of the neuron that carries each edge.
 *
 * The calls follow Algorithm 1's statement of the problem: INPUT an implicit function built
 * from a ReLU MLP (am_load_mlp), a trigger point on the surface (am_seed, Alg. 1 step 2 and
 * Sec. 4.3), OUTPUT the polygon mesh Z = {V, {P}} (am_march, am_get_mesh).
 *
 * Conventions shared by every call:
 *   - every call returns an am_status and never aborts the process; on failure
 *     am_last_error() describes the cause;
 *   - pointers named h_* are HOST pointers, d_* are DEVICE pointers of the context's
 *     device; the library copies every input it is given, so inputs may be freed as soon
 *     as the call returns; output buffers stay owned by the caller;
 *   - all device work runs on the context's stream; calls are blocking with respect to
 *     that stream unless stated otherwise;
 *   - there is no CPU fallback: without a usable CUDA device am_create fails.
 *
 * Conventions of the data (identical in the CPU oracle):
 *   - biases are kept: every affine map is a row [a_x a_y a_z | a_0] acting on [x; 1];
 *   - a cell key holds one bit per hidden neuron, in layer order, bit k of neuron k at
 *     64-bit word k / 64, bit k % 64; the state is 1 iff the pre-activation is > 0 (a tie
 *     gives 0, Eq. 2);
 *   - faces are clipped to the box [-B, B]^3; edges on the box carry the plane ids
 *     N + 0..5 for the box faces +x, -x, +y, -y, +z, -z (N = number of hidden neurons);
 *   - a face's vertices run counter-clockwise seen from +grad F (= a_F[0:3]);
 *     edge_planes[i] is the plane carrying the edge from corner i to corner i + 1;
 *   - a mesh vertex is identified by the key (i, j, s with bits i and j cleared), i < j the
 *     two planes meeting there, so the up to four faces meeting at a vertex share it.
 */
#ifndef ANALYTIC_MARCHING_H
#define ANALYTIC_MARCHING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct am_ctx am_ctx;

typedef enum {
    AM_OK = 0,
    AM_ERR_INVALID_ARG = 1,   /* a NULL pointer, a size out of range, an unknown net id */
    AM_ERR_CUDA = 2,          /* a CUDA runtime call failed; the context may be unusable */
    AM_ERR_CAPACITY = 3,      /* a cell, hash, vertex or per-face vertex capacity was exceeded */
    AM_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up */
    AM_ERR_NO_SEED_CELL = 5,  /* no ray produced a seed cell (no sign change / no common cell) */
    AM_ERR_DEGENERATE = 6,    /* the walk met a face it could not clip (reported, not fatal) */
    AM_INCOMPLETE = 7,        /* am_march stopped at max_cells; call it again to resume */
    AM_ERR_STATE = 8          /* the call is not valid in the context's current state */
} am_status;

typedef enum {
    AM_PREC_FP64 = 0,         /* compose and clip in FP64 (the plain path) */
    AM_PREC_MIXED = 1,        /* compose in double-float arithmetic on the FP32 pipes with a
                                 rigorous error bound per row; vertices solved in FP64; every
                                 sign test certified against the bounds (FP32, then FP64 for
                                 close calls); a cell with an undecidable test is redone in FP64 */
    AM_PREC_TENSOR = 2,       /* am_compose only, kept as the measured baseline that AM_PREC_SLICED
                                 replaces (legacy mma.sync, not tcgen05): the hidden layers on the
                                 tensor cores, W and Z
                                 split into three BF16 parts, four mma.sync products per tile
                                 accumulated in FP32 (about 1e-6 relative); each row carries an
                                 error ESTIMATE (random-sign model of the accumulation with a
                                 safety factor 8, root-mean-square propagation), not a bound, so
                                 am_march refuses it.  Needs 32 ceil(n_{l-1} / 16) <= max_neurons
                                 + 10 for l >= 2. */
    AM_PREC_SLICED = 3        /* the hidden layers on the tcgen05 tensor cores as error-free BF16 digit
                                 products (Ozaki scheme): W_l and each cell's masked Z_{l-1} are split
                                 into 8 planes of 6-bit integer digits with a power-of-two scale per
                                 row / column; every plane product and its FP32 accumulation is exact,
                                 and the diagonals are combined in 64-bit integers, then FP64.  The
                                 rows are FP64-class (error <= (3 n_{l-1} + 1) 2^-48 times the row
                                 and column scales, the order of an FP64 dot product's worst case);
                                 many cells share each weight tile.  Needs n_{l-1} <= 1638. */
} am_precision;

typedef enum {
    AM_SCHED_PERSISTENT = 0,  /* one launch: resident blocks take cells from a ticket queue */
    AM_SCHED_LEVELS = 1       /* one launch per breadth-first level, synchronised by the host */
} am_schedule;

/* Rows a cell's face is clipped with before the all-row check (which keeps the result exact
 * whatever the candidates are: any violated row is cut in and the check repeated). */
typedef enum {
    AM_CAND_NEAREST = 0,      /* the 32 rows nearest to the point the cell was entered through */
    AM_CAND_LEARNED = 1,      /* the 32 rows the learned proposal scores highest (am_proposal_*);
                                 nets whose N or depth do not match the proposal fall back to
                                 AM_CAND_NEAREST */
    AM_CAND_NONE = 2          /* no candidates: the all-row check clips alone (the plain clip) */
} am_candidates;

/* Context creation options.  Zero-initialised fields take the documented defaults. */
typedef struct {
    int device;               /* CUDA device ordinal (default 0) */
    void *stream;             /* cudaStream_t to run on; NULL = a stream owned by the context */
    int64_t max_cells;        /* capacity of visited cells over all nets (default 1 << 20) */
    int64_t hash_slots;       /* cell hash-table slots, rounded up to a power of two
                                 (default: the power of two >= 2 * max_cells) */
    int max_face_verts;       /* per-face vertex capacity, 8..62 (default 32) */
    int max_neurons;          /* largest N of any net that will be loaded (default 4096) */
    int max_width;            /* largest hidden width of any net that will be loaded (default 512) */
} am_ctx_opts;

/* One ReLU MLP (Sec. 2.2, Eq. 1 with biases): F(x) = w_out . h_L + b_out,
 * h_l = relu(W_l u_l + b_l + S_l h_src(l)); u_1 = [x; z]; u_l = h_{l-1}, or concat(h_{l-1}, [x; z])
 * at the skip layer (a DeepSDF-style skip-concat shortcut, Sec. 5.1); h_0 = x.  The optional
 * residual shortcut S_l h_src(l) is Sec. 5.1's residual block ending at layer l: the identity
 * (first kind, g(x + T x)) or a matrix V (second kind, g(V x + T x)) from an earlier layer.
 * Row-major FP64, caller owned, copied by am_load_mlp. */
typedef struct {
    int latent_dim;           /* length of the fixed latent code z (0 = none) */
    const double *latent;     /* z, latent_dim values (may be NULL when latent_dim == 0) */
    int n_hidden;             /* L >= 1 */
    const int *width;         /* n_1..n_L */
    const double *const *W;   /* W_l: width[l] x fan_in(l); fan_in(1) = 3 + latent_dim;
                                 fan_in(l) = width[l-1] (+ 3 + latent_dim at the skip layer) */
    const double *const *b;   /* b_l: width[l] */
    int skip_layer;           /* 0 = none, else the 1-based hidden layer taking the concat */
    const double *w_out;      /* width[L] */
    double b_out;
    double slope;             /* the hidden activation g(a) = a for a > 0, slope * a otherwise: 0 = ReLU,
                                 else a leaky / parametric ReLU (the paper's closing remarks).  The
                                 cells are Def. 2's either way; inside a cell the masks diag(s_l) of
                                 Cor. 1 become diag(s_l + slope (1 - s_l)).  |slope| < 1; such nets
                                 march in FP64 (AM_PREC_MIXED falls back to it; AM_PREC_SLICED and
                                 am_compose other than FP64 refuse them) */
    const int *shortcut_src;  /* NULL, or n_hidden entries: hidden layer l (1-based, entry l - 1) adds
                                 S_l h_src to its pre-activation, src in 0 .. l - 1 (0 = the input x,
                                 3 coordinates; >= 1 a hidden layer), or -1 for none.  A shortcut
                                 from x is folded into the layer's constant rows at load time;
                                 a net with a shortcut from a hidden layer marches in FP64, as a
                                 leaky net does */
    const double *const *shortcut_S;   /* NULL, or n_hidden pointers: S_l, width[l] x n_src row-major
                                 (n_src = 3 for x, else width[src]); a NULL pointer = the identity,
                                 which needs n_src == width[l] */
    int n_heads;              /* 0 or 1: one output (w_out, b_out).  M = n_heads in 2..AM_MAX_HEADS: a
                                 final max pooling (Sec. 5.2), F = max_i (w_heads[i] . h_L + b_heads[i]),
                                 w_out and b_out unused.  M sub-networks sit side by side in the hidden
                                 layers (block-diagonal W_l, the caller's layout) and head i reads its
                                 sub-network's last layer.  A cell is a unit pattern together with the
                                 index j of the pooled maximum (the first on a tie); its face lies on
                                 head j's plane a_F(j) and its system gains the pooling rows
                                 a_F(i) - a_F(j) (i != j) as planes N_units + i, so the net has
                                 N = N_units + M plane ids and key bits (j one-hot in the last M),
                                 and the box planes are N + 0..5.  Crossing pooling plane N_units + i
                                 moves the maximum to i.  Pooled nets march in FP64 */
    const double *w_heads;    /* n_heads x width[L] (n_heads >= 2) */
    const double *b_heads;    /* n_heads */
} am_mlp_desc;
#define AM_MAX_HEADS 64

/* Options of one march. */
typedef struct {
    double box;               /* B of the clip box [-B, B]^3 (default 1.5) */
    double delta;             /* vertex tolerance in world units (default 1e-10): a plane within
                                 delta of a vertex counts as satisfied and as a degenerate event */
    am_precision precision;   /* AM_PREC_FP64 (default), AM_PREC_MIXED or AM_PREC_SLICED (one net per
                                 context; level schedule: per batch of a level's cells the rows are
                                 composed on the tensor cores into device memory, then clipped in FP64) */
    int64_t max_cells;        /* stop after this many cells have been solved (0 = no limit) */
    am_candidates candidates; /* AM_CAND_NEAREST (default), AM_CAND_LEARNED or AM_CAND_NONE */
    am_schedule schedule;     /* AM_SCHED_PERSISTENT (default) or AM_SCHED_LEVELS */
    int grid_blocks;          /* persistent schedule: blocks to launch (0 = all resident) */
} am_march_opts;

/* Statistics of the last march (cumulative over resumed calls). */
typedef struct {
    int64_t cells;            /* cells solved */
    int64_t faces;            /* non-empty faces */
    int64_t empty_faces;      /* cells whose face was empty or of zero area */
    int64_t vertices;         /* assembled (deduplicated) vertices */
    int64_t corners;          /* face corners (sum of face sizes) */
    int64_t degenerate;       /* planes within delta of an accepted vertex */
    int64_t open_faces;       /* faces with an edge on the box */
    int64_t refined_cells;    /* mixed precision: cells solved in FP64, because a sign test could not
                                 be certified or because the net is too deep and wide for the
                                 double-float bound (decided per net at load time) */
    int64_t levels;           /* breadth-first levels marched */
    double ms_march;          /* device time of the march (CUDA events) */
    double ms_assemble;       /* device time of the mesh assembly */
    double ms_cell_kernels;   /* summed device time of the cell-solving kernel launches */
    int64_t cell_launches;    /* launches of the cell-solving kernel */
    int64_t kernel_launches;  /* all kernel launches of the library since the last am_reset */
    int64_t close_calls;      /* mixed precision: sign tests re-evaluated in FP64 */
    int64_t fixups;           /* faces whose candidate polygon the all-row check corrected */
    int64_t cuts;             /* half-plane cuts applied to face polygons (candidates + corrections) */
    int64_t phase_cycles[10]; /* SM cycles summed over cells per phase (compose, set-up, candidate
                                 sort, candidate clip, FP64 vertices, check, emit, march, waiting
                                 for work, spare); only filled by a build with -DAM_PHASE_TIMERS,
                                 zero otherwise */
    double ms_compose;        /* AM_PREC_SLICED march: device time of the tensor-core compose launches */
    double ms_clip;           /* AM_PREC_SLICED march: device time of the clip launches reading those rows */
    double ms_proposal;       /* AM_PREC_SLICED march with AM_CAND_LEARNED: device time of the proposal's
                                 forward pass on the tensor cores (features and three products per batch) */
    int64_t clip_fallbacks;   /* AM_PREC_SLICED march: cells the warp-per-cell clip handed to the block
                                 kernel (a test it could not decide outright, a large polygon) */
    int64_t tensor_macs;      /* AM_PREC_SLICED: BF16 multiply-adds the compose issued on the tensor cores
                                 (36 digit-plane products per layer over the padded tiles) */
} am_stats_t;

/* Assembled mesh of one net.  Two-call protocol for am_get_mesh: with every array pointer
 * NULL the call only fills the counts; with non-NULL arrays (host memory, sized from the
 * counts) it copies the mesh out. */
typedef struct {
    int64_t n_vertices;
    int64_t n_faces;
    int64_t n_corners;        /* sum of the face sizes */
    int key_words;            /* 64-bit words per face key */
    int64_t n_open_faces;
    double *xyz;              /* 3 * n_vertices */
    int64_t *face_offsets;    /* n_faces + 1; face f is corners [off[f], off[f+1]) */
    int32_t *face_vertices;   /* n_corners vertex indices */
    int32_t *edge_planes;     /* n_corners plane ids (edge corner i -> corner i+1) */
    uint64_t *face_keys;      /* n_faces * key_words */
} am_mesh;

/* Create a context on opts->device (opts may be NULL for defaults).  Allocates every device
 * buffer up front, sized by the capacities.  Returns AM_ERR_CUDA when no device is usable. */
am_status am_create(am_ctx **ctx, const am_ctx_opts *opts);

/* Free the context and all of its device memory.  NULL is ignored. */
void am_destroy(am_ctx *ctx);

/* Text of the last error of this context (static storage owned by the context). */
const char *am_last_error(const am_ctx *ctx);

/* Copy one MLP to the device (Sec. 2.2).  The skip concat and the latent code are folded
 * into per-layer constant affine rows at load time.  *net_id receives the id used by
 * am_seed / am_get_mesh.  Fails with AM_ERR_INVALID_ARG when the net exceeds max_neurons
 * or max_width. */
am_status am_load_mlp(am_ctx *ctx, const am_mlp_desc *desc, int *net_id);

/* Forget all cells, faces and seeds of every net (the loaded nets stay). */
am_status am_reset(am_ctx *ctx);

/* Forget all cells and faces (as am_reset) and free every loaded net; net ids restart at 0. */
am_status am_release_nets(am_ctx *ctx);

/* Trigger (Alg. 1 step 2; dichotomy, Sec. 4.3.2): for each ray x(t) = o + t d, t in [0, R],
 * bisect F on the device until both ends of the bracket lie in one cell, take the exact
 * affine root in that cell and push its cell into the active set.  h_origins, h_dirs: host,
 * n_rays x 3 FP64.  *n_seeded (may be NULL) receives the number of new seed cells (rays
 * landing in an already seeded cell count once).  AM_ERR_NO_SEED_CELL when no ray
 * produced one.  F and the patterns are evaluated in double-float arithmetic (FP32 pairs,
 * about 44 bits) for nets without hidden shortcuts, pooling or leaky units, else in FP64: a
 * sign or a pattern bit can differ from an FP64 evaluation only within about 1e-12 of zero. */
am_status am_seed(am_ctx *ctx, int net_id, const double *h_origins, const double *h_dirs,
                  int n_rays, double R, int *n_seeded);

/* Trigger by sphere tracing for an SDF (Sec. 4.3.1): from each start point x_0 (h_starts:
 * host, n_starts x 3 FP64) the device walks x <- x - eta F(x) grad F(x), grad F being the
 * gradient of the affine piece of the cell x lies in (a tie gives state 0), until
 * |F(x)| <= eps or max_steps steps.  Through the last point x_T it then bisects (as am_seed)
 * the segment x_T + s n, |s| <= h, n = grad F / |grad F|, h = 2|F(x_T)|/|grad F| + 1e-9,
 * which brackets the zero crossing of x_T's cell, and pushes the cell found.  Start points
 * whose walk meets a cell with grad F = 0, or whose segment has no sign change, produce no
 * seed.  0 < eta <= 1; 0 <= max_steps <= 65536; eps >= 0; 1 <= n_starts <= 2^24.
 * *n_seeded (may be NULL): new seed cells.  h_seed_points (host, n_starts x 3, may be NULL):
 * each start's seed point, NaN where it produced none.  AM_ERR_NO_SEED_CELL when no start
 * produced a new cell. */
am_status am_seed_sphere_trace(am_ctx *ctx, int net_id, const double *h_starts, int n_starts, double eta,
                               int max_steps, double eps, int *n_seeded, double *h_seed_points);

/* Trigger by random-pair dichotomy (Sec. 4.3.2): F is evaluated on the device at every sample
 * (h_points: host, n_points x 3 FP64, drawn by the caller; in the precision am_seed states); the r-th sample with F < 0 is
 * paired with the r-th sample with F > 0, in sample order, for r < min(#negative, #positive,
 * max_pairs) (samples with F == 0 are not used); each pair's segment from x- to x+ is bisected
 * as in am_seed and its cell pushed.  1 <= n_points, max_pairs <= 2^24.  *n_pairs and
 * *n_seeded (may be NULL): pairs formed and new seed cells.  h_seed_points (host, max_pairs x 3,
 * may be NULL): the seed point of pair r in row r, NaN where it produced none and in the rows
 * past the last pair.  AM_ERR_NO_SEED_CELL when no pair formed or none produced a new cell. */
am_status am_seed_pairs(am_ctx *ctx, int net_id, const double *h_points, int n_points, int max_pairs,
                        int *n_pairs, int *n_seeded, double *h_seed_points);

/* March (Alg. 1): solve every active cell (compose its affine maps, clip its face, push its
 * unseen neighbours), breadth first over all nets at once, then assemble the meshes.
 * opts may be NULL for defaults.  AM_INCOMPLETE when opts->max_cells stopped it early. */
am_status am_march(am_ctx *ctx, const am_march_opts *opts);

/* Copy out the assembled mesh of one net (two-call protocol, see am_mesh). */
am_status am_get_mesh(am_ctx *ctx, int net_id, am_mesh *mesh);

/* Device view of the assembled mesh of one net, without a copy (Alg. 1 output).  The array
 * pointers of *mesh receive DEVICE addresses inside the context's own assembly buffers, in the
 * layout am_get_mesh copies out (face_offsets start at 0 for this net; corner vertex indices
 * refer to this net's xyz).  The arrays stay owned by the context and valid until the next
 * am_march, am_reset, am_release_nets or am_destroy; the caller must not write or free them.
 * The call synchronises the context's stream before it returns.  n_open_faces is set to -1
 * (not computed here; am_get_mesh computes it). */
am_status am_get_mesh_device(am_ctx *ctx, int net_id, am_mesh *mesh);

/* Canonical order of a host mesh (as filled by am_get_mesh), in place; no context, no device.
 * Alg. 1 leaves the order of the faces to the march, and the device's breadth-first discovery
 * is not deterministic; this order is:
 *   faces ascending by cell key read as an N-bit unsigned integer (face_keys word key_words-1
 *     is the most significant);
 *   each face's ring (face_vertices and edge_planes together, orientation kept) starts at the
 *     corner whose sorted pair of plane ids (the edge into it, the edge out of it) is smallest;
 *   vertices numbered by first appearance along that corner sequence (xyz permuted to match;
 *     vertices no face uses, if any, follow in their old order).
 * The same surface therefore gives the same arrays, whatever order the march found it in.
 * AM_ERR_INVALID_ARG for inconsistent arrays (offsets not rising from 0 to n_corners, a face
 * with fewer than 3 corners, a vertex index out of range). */
am_status am_mesh_canonicalize(am_mesh *mesh);

/* Fan triangulation of a host mesh (Sec. 4.4: each convex face splits along diagonals into
 * V - 2 triangles): face (v_0 ... v_{V-1}) gives (v_0, v_j, v_{j+1}), j = 1 .. V-2, in face
 * order, so the triangles keep the face's orientation.  Two-call protocol: with tri NULL,
 * *n_tri receives the count (n_corners - 2 n_faces); otherwise tri (host, 3 x *n_tri int32) is
 * filled and AM_ERR_CAPACITY is returned when *n_tri is smaller than the count. */
am_status am_mesh_triangulate(const am_mesh *mesh, int32_t *tri, int64_t *n_tri);

/* Statistics of the last march. */
am_status am_get_stats(const am_ctx *ctx, am_stats_t *stats);

/* Test hook for the time-out path; no counterpart in the paper.  Every wait of the persistent
 * march for work is bounded (4 s by default): a block that waits longer sets the time-out
 * status and returns, and am_march then returns AM_ERR_TIMEOUT without assembling a mesh.
 * This call makes the next am_march exercise that path without faulting or hanging the GPU:
 * before its launch, `unpublished_ids` cell ids (1 <= unpublished_ids <= max_cells) are handed
 * out that no block ever publishes, as if the blocks that claimed them had stopped, and every
 * wait for work gives up after wait_limit_ms (0 < wait_limit_ms <= 4000).  The setting applies
 * to the next am_march only, which must use the persistent schedule (AM_ERR_INVALID_ARG
 * otherwise).  After any AM_ERR_TIMEOUT the context refuses am_seed and am_march
 * (AM_ERR_STATE) until am_reset, which also clears a pending stall. */
am_status am_test_stall_next_march(am_ctx *ctx, int64_t unpublished_ids, double wait_limit_ms);

/* Compose only (Lemma 1, Cor. 1; Eq. 10): the affine rows of the cells whose activation
 * patterns are d_keys (device, n x ceil(N/64) words, bit k = state of neuron k), for net_id, in
 * the given precision.  d_rows (device, n x (N + 1) x 4 doubles) receives for each key the N
 * sign-adjusted rows (1 - 2 s_k) [a_k | a_k0] of Eq. 10 followed by [a_F | a_F0] (Eq. 8);
 * d_err (device, n x (N + 1) floats, may be NULL) the per-row error bound (AM_PREC_MIXED),
 * estimate (AM_PREC_TENSOR) or 0 (AM_PREC_FP64, AM_PREC_SLICED), as an l1 bound on the 4
 * coefficients.  AM_PREC_SLICED composes the patterns in batches (the context allocates its
 * scratch on first use) and returns AM_ERR_TIMEOUT if a tensor-core pipeline wait gave up. */
am_status am_compose(am_ctx *ctx, int net_id, const uint64_t *d_keys, int64_t n, am_precision precision,
                     double *d_rows, float *d_err);

/* Rank-1 neighbour compose (Cor. 1 across one flipped neuron; Alg. 1 step 10): the rows of the n
 * cells key(parent i) XOR e_{flip[i]} from their parents' rows.  Crossing the plane of neuron k of
 * layer l leaves Z_1..Z_l unchanged (the sign of row k flips with its state), and for j > l Z_j
 * changes by the rank-1 term v_j a^T: a = the parent's signed row k, v_{l+1} = W_{l+1}[:, k],
 * v_j = W_j diag(s_{j-1}) v_{j-1}; a_F by (w_out . diag(s_L) v_L) a (w_out[k] a when l = L).  The
 * products run on the tcgen05 tensor cores as in AM_PREC_SLICED, with one operand column per
 * cell instead of four.  This is the compose the AM_PREC_SLICED march uses for most cells (see
 * am_tuning.rank1_period); this call exposes it on caller arrays:
 *   d_parent_keys  n x ceil(N/64) words, the parents' activation patterns (device)
 *   d_parent_rows  n x (N + 1) x 4 doubles, the parents' rows as am_compose writes them (device)
 *   d_flip         n neuron ids in [0, N), the neuron each child flips (device)
 *   d_rows         out: n x (N + 1) x 4 doubles, the children's rows in am_compose's layout (device)
 * The parents' rows are taken to 48 bits (FP32 pairs, the march's representation) on input.
 * Synchronous; allocates its scratch per call.  AM_ERR_INVALID_ARG for a flip outside [0, N) or a
 * net whose fan-ins exceed the sliced path's limit; AM_ERR_TIMEOUT if a tensor-core pipeline wait
 * gave up. */
am_status am_compose_neighbors(am_ctx *ctx, int net_id, const uint64_t *d_parent_keys, const double *d_parent_rows,
                               const int32_t *d_flip, int64_t n, double *d_rows);

/* ---- launch shapes and autotuning --------------------------------------------------------
 * No counterpart in the paper: these calls change how fast a result is computed, never the
 * result.  Kernels with more than one valid launch shape read it from the context;
 * am_set_tuning sets it by hand, am_autotune_compose times every candidate and keeps the
 * fastest.  am_autotune_march picks the march's precision and schedule, all of which give the
 * same faces, edge cycles and vertex identities (vertex coordinates agree to rounding). */
typedef struct {
    int compose_tile_cells;   /* AM_PREC_SLICED: cells stacked per tensor-core tile: 32 (UMMA N = 128,
                                 the 8 diagonals in two passes of 4), 16 (N = 64, all 8 diagonals
                                 at once, one tile per SM) or 8 (N = 32, two tiles per SM);
                                 0 (default) = automatic per batch and layer: the 32-cell tile
                                 when n_{l-1} > 448 (8 K chunks) and its tiles, split over up to
                                 4 K ranges, fill every SM, else the 16-cell tile */
    int rank1_period;         /* AM_PREC_SLICED march: a cell entered across neuron k of layer l keeps its
                                 parent's rows Z_1..Z_l and gets Z_{l+1..L} and a_F by a rank-1 update
                                 from the parent's rows (one operand column instead of four, Cor. 1);
                                 every rank1_period-th generation of a chain is composed in full,
                                 which bounds the rounding the updates accumulate.  1 = always in
                                 full; 0 (default) = 32 */
    int clip_kernel;          /* AM_PREC_SLICED march with candidates: 0 (default) = one warp per cell for
                                 every cell whose tests it decides outright, the block kernel for the
                                 rest; 1 = the block kernel (one block per cell) for every cell */
    int check_kernel;         /* AM_PREC_SLICED march, clip_kernel 0: the dense check of every row at
                                 every vertex (Eq. 10) after the candidate clip.  0 (default) = in
                                 the warp clip, certified FP32 on the CUDA cores; 1 = on the tcgen05
                                 tensor cores for polygons of at most 16 vertices (each 128-row tile
                                 of the cell's rows times its vertices, exact BF16 parts, FP32
                                 accumulators, a certified sign test with FP64 close calls), any
                                 violated row sending the cell to the block kernel.  Both give the
                                 same mesh. */
} am_tuning;

/* Set (t != NULL) the context's launch shapes.  AM_ERR_INVALID_ARG for an unsupported value. */
am_status am_set_tuning(am_ctx *ctx, const am_tuning *t);

/* The context's current launch shapes. */
am_status am_get_tuning(const am_ctx *ctx, am_tuning *t);

/* One timed candidate of the autotuner. */
typedef struct {
    int compose_tile_cells;   /* the candidate's cells per tensor-core tile */
    float ms;                 /* median device time of one am_compose(AM_PREC_SLICED) call */
} am_tune_point;

/* Autotuner of the sliced tensor-core compose (K-stacking tile shape).  For every supported
 * compose_tile_cells (the automatic choice 0 included) it runs am_compose(AM_PREC_SLICED) of the n patterns d_keys (device,
 * n x ceil(N/64) words) of net_id into d_rows (device, n x (N + 1) x 4 doubles) once untimed,
 * then `reps` times between CUDA events on the context's stream; it keeps the candidate with
 * the smallest median in the context (as am_set_tuning would; a later candidate must be more
 * than 1 % faster than an earlier one, and the automatic choice is tried first) and writes every candidate, in
 * the order tried, to h_points (host, at most max_points entries; *n_points receives how many
 * were tried).  Every candidate computes the same rows bit for bit; only the time differs.
 * The best shape depends on the batch size: tune on batches of the size that will be composed
 * (for AM_PREC_SLICED marches, one breadth-first level: typically a few hundred cells). */
am_status am_autotune_compose(am_ctx *ctx, int net_id, const uint64_t *d_keys, int64_t n, double *d_rows, int reps,
                              am_tune_point *h_points, int max_points, int *n_points);

/* One timed candidate of the march autotuner. */
typedef struct {
    am_precision precision;
    am_schedule schedule;
    float ms;                 /* median device time of am_march over the repetitions */
} am_march_point;

/* Autotuner of the march's execution path.  Every precision and schedule gives the same faces
 * and connectivity (coordinates agree to rounding), so the choice is a matter of time.  For each candidate (FP64 and mixed precision, each
 * with the persistent and the level schedule, and AM_PREC_SLICED when the context holds this
 * one net and its fan-ins allow it), it marches net_id from the given rays (as am_seed; host
 * arrays, n_rays x 3) up to max_cells cells (0 = the whole mesh), `reps` times after one untimed
 * run, timing each am_march with its CUDA events.  *best (in/out): its other fields (box,
 * delta, candidates, grid_blocks) are used as given; precision and schedule are set to the
 * fastest candidate's.  h_points (host, may be NULL) receives up to max_points candidates in
 * the order tried; *n_points (may be NULL) how many were tried.  Ends with am_reset: the
 * context holds no cells afterwards. */
am_status am_autotune_march(am_ctx *ctx, int net_id, const double *h_origins, const double *h_dirs, int n_rays,
                            double R, int64_t max_cells, int reps, am_march_opts *best, am_march_point *h_points,
                            int max_points, int *n_points);

/* ---- learned constraint proposal --------------------------------------------------------
 * No counterpart in the paper.  A small MLP, x (7 + L) -> H -> H -> n_out, ReLU hidden layers,
 * sigmoid scores, that predicts which of the n_out = N neurons of a net carry the edges of a
 * cell's face.  Features of a cell: the point it was entered through (3), the unit normal of its
 * face plane a_F[0:3] / |a_F[0:3]| (3), the plane offset a_F[3] / |a_F[0:3]| (1), and the active
 * fraction of each hidden layer (L).  Parameters are one flat FP32 array, in this order:
 * W1 (H x n_in), b1 (H), W2 (H x H), b2 (H), W3 (n_out x H), b3 (n_out), matrices row-major.
 * Training uses BF16 operands with FP32 accumulation and Adam on FP32 master weights. */

/* Training samples from the mesh of net_id assembled by the last am_march (labels are what the
 * march found, so they are exact whatever candidates it used): one sample per corner of every
 * face, in the assembled face order; the entry point of a sample is the midpoint of the edge that
 * leaves its corner, the plane is the face's (Newell normal of its vertices).  Writes
 * n = min(corners, max_samples) rows of d_X (n x (7 + L) FP32, device) and d_Y (n x N FP32 0/1,
 * device) and returns n in *n_samples; with d_X or d_Y NULL only *n_samples is set. */
am_status am_proposal_samples(am_ctx *ctx, int net_id, float *d_X, float *d_Y, int64_t max_samples,
                              int64_t *n_samples);

/* Create (or replace) the context's proposal with Kaiming-normal weights drawn from seed.
 * max_batch bounds the samples of one forward / gradient call.  n_in <= 64; hidden is even and
 * <= 768 (the march evaluates the proposal in shared memory with BF16-pair loads). */
am_status am_proposal_init(am_ctx *ctx, int n_in, int hidden, int n_out, int max_batch, uint64_t seed);

/* Copy the flat FP32 parameters out of / into the context (host arrays of n_params values). */
am_status am_proposal_get_params(am_ctx *ctx, float *h_params, int64_t n_params);
am_status am_proposal_set_params(am_ctx *ctx, const float *h_params, int64_t n_params);

/* Logits of n samples: d_X (n x n_in FP32, device) -> d_Z (n x n_out FP32, device). */
am_status am_proposal_forward(am_ctx *ctx, const float *d_X, int n, float *d_Z);

/* Mean binary cross-entropy of n <= max_batch samples (labels d_Y, n x n_out, 0/1 FP32,
 * device) and its gradient w.r.t. every parameter (host array of n_params values). */
am_status am_proposal_grad(am_ctx *ctx, const float *d_X, const float *d_Y, int n, float *h_grads,
                           int64_t n_params, float *h_loss);

/* steps Adam steps (learning rate lr) on minibatches of `batch` consecutive samples, cycling
 * through the n samples of d_X / d_Y (device).  h_losses (host, may be NULL) receives the loss
 * of each step. */
am_status am_proposal_train(am_ctx *ctx, const float *d_X, const float *d_Y, int64_t n, int batch, int steps,
                            float lr, float *h_losses);

/* ---- allocation-free vertex assignment ---------------------------------------------------
 * The paper has no counterpart to this call; it serves callers that cannot allocate device
 * memory.  Code captured into a CUDA graph cannot call cudaMalloc, and some host frameworks
 * hand out every device byte from their own pool.  Such callers can still build the mesh's
 * vertex indices from faces they hold.
 *
 * For every corner of n_faces analytic faces it writes the index of the corner's mesh vertex,
 * the same grouping as am_march's assembly: corners share an index exactly when their
 * combinatorial vertex keys (i, j, s with bits i and j cleared) are equal.  The faces use the
 * layout am_get_mesh returns:
 *   d_face_keys      n_faces x key_words cell keys (device)
 *   d_face_offsets   n_faces + 1 corner offsets, d_face_offsets[0] == 0 (device)
 *   d_edge_planes    n_corners plane ids, edge corner c -> corner c + 1 (device)
 *   n_neurons        N of the net; plane ids >= N (the box) carry no key bit.  A max-pooled net's
 *                    pooling planes are not named by their pair of heads here (am_get_mesh's
 *                    assembly does that): pass its faces to am_get_mesh instead
 *   d_corner_vertex  out: n_corners vertex indices in [0, *d_n_vertices) (device)
 *   d_n_vertices     out: one int64, the number of distinct vertices (device); NEGATIVE when some
 *                    corner got no vertex: -1 a face has more than AM_NOALLOC_MAX_FACE_CORNERS
 *                    corners or offsets outside [0, n_corners] (the corners of a face that is
 *                    only too long are set to -1), -2 a hash probe gave up (that corner is -1),
 *                    -3 both; the indices are then not a valid grouping
 *   stream           cudaStream_t of the caller (NULL = the legacy default stream); the call is
 *                    asynchronous on it, so errors found by the kernels arrive through
 *                    *d_n_vertices, not through the return value
 * Vertex indices are numbered in no particular order.  A face may have at most
 * AM_NOALLOC_MAX_FACE_CORNERS (62) corners, as am_march's faces (max_face_verts <= 62).
 *
 * It allocates nothing: no cudaMalloc, cudaFree or allocating library routine.  Its scratch
 * memory is one file-scope device table of 2^22 hash slots (32 MiB) that every GPU loading the
 * library keeps until the process exits.  The first call on a device looks up the table's
 * device address with that device current; make that first call before any stream capture.
 * Every call shares the table and clears the part it uses, so calls whose work overlaps on the
 * GPU (two streams, or two host threads) race and give wrong results: serialise them.
 * Returns AM_ERR_CAPACITY when n_corners > 2^21 (AM_NOALLOC_MAX_CORNERS), AM_ERR_INVALID_ARG
 * for a NULL pointer or a negative size, AM_ERR_CUDA when no device is current or a launch
 * fails. */
#define AM_NOALLOC_MAX_CORNERS ((int64_t)1 << 21)
#define AM_NOALLOC_MAX_FACE_CORNERS 62
am_status am_assign_vertices_noalloc(const uint64_t *d_face_keys, int key_words,
                                     const int64_t *d_face_offsets, const int32_t *d_edge_planes,
                                     int64_t n_faces, int64_t n_corners, int n_neurons,
                                     int32_t *d_corner_vertex, int64_t *d_n_vertices, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ANALYTIC_MARCHING_H */
