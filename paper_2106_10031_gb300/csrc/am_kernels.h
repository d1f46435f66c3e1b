// am_kernels.h -- launch interface between the host library (am_api.cu) and the kernels.
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "am_common.cuh"

namespace am {

// candidate rows clipped before the all-row check
enum { kCandNearest = 0, kCandLearned = 1, kCandNone = 2 };

// the learned proposal as the march reads it (BF16 weights, W2 and W3 transposed)
struct ProposalView {
    const __nv_bfloat16 *w1;      // hidden x n_in
    const float *b1;              // hidden
    const __nv_bfloat16 *w2t;     // hidden x hidden, [in][out]
    const float *b2;
    const __nv_bfloat16 *w3t;     // hidden x (n_out rounded up to even), [in][out]
    const float *b3;
    int n_in, hidden, n_out;
};

struct CheckRec;
struct MarchArgs {
    const NetDev *nets;
    Arena ar;
    double box, delta;
    float box_hi, box_lo;    // box as an FP32 pair (box_hi + box_lo == box), set on the host with box
    int max_n, max_w;        // shared-memory sizing (largest loadable net)
    long long limit;         // persistent schedule: tickets >= limit are not solved
    long long wait_ns;       // persistent schedule: limit on any wait for work (ns)
    int64_t begin, end;      // level schedule: cell ids solved by this launch
    int candidates;          // kCandNearest / kCandLearned / kCandNone
    int tc;                  // compose only (mode 1): hidden layers composed on the tensor cores
    ProposalView prop;       // used with kCandLearned for nets with N == prop.n_out
    const void *rows_in;     // level schedule: rows of cells [begin, end) composed beforehand on the
                             // tensor cores, n x (N + 1) FP32 pairs, a_F last: per cell the N + 1 hi
                             // words [hi x 4], then the N + 1 lo words [lo x 4]
    const __nv_bfloat16 *scores_in;   // level schedule, learned candidates: the proposal's scores of
    int scores_ld;                    // cells [begin, end), scores_ld BF16 per cell, from the tensor cores
    const int32_t *list;              // level schedule: solve the cells list[0 .. *list_count) (ids in
    const unsigned long long *list_count;   // [begin, end)) instead of the whole range
    int32_t *fb_list;                 // warp clip: cells it hands to the block kernel, and their count
    unsigned long long *fb_count;
    unsigned long long *work;         // warp clip: zero before the launch; the warps take cells begin + the
                                      // counter's next value (null: a fixed stride over a one-warp-per-cell grid)
    CheckRec *chk;                    // warp clip with the dense check on the tensor cores: the clipped
    unsigned long long *chk_count;    // polygons it hands to check_tc (null: the warp checks them itself)
    const int *chk_status;            // finish pass: per record 0 = every row holds, else the block kernel
};
// A polygon the warp clip hands to the dense check (am_check_tc.cu): the cell, its m <= kChkMaxV
// vertices (FP64) and the plane of each edge (edge i: vertex i -> i + 1).
constexpr int kChkMaxV = 16;
struct CheckRec {
    int32_t cell, m;
    int32_t pe[kChkMaxV];
    double v[kChkMaxV][3];
};
// the sliced level march's clip, one warp per cell (am_clip_warp.cu): cells [begin, end), rows in
// rows_in; cells it cannot decide are appended to fb_list for march_range_kernel (list mode).
// With a.chk set, polygons of at most kChkMaxV vertices are not checked here but appended to
// a.chk; after check_tc, launch_clip_warp_finish emits and pushes the records whose status is 0
// and hands the others to fb_list.
cudaError_t prepare_clip_warp();
void launch_clip_warp(const MarchArgs &a, cudaStream_t st);
void launch_clip_warp_finish(const MarchArgs &a, cudaStream_t st);
// The dense all-constraint check on the tcgen05 tensor cores: for every record, every neuron row
// of its cell (FP32 pairs in rows, cell c at rows + (c - begin) 8 (N + 1) floats) at every vertex,
// as the products [rows x K] . [K x 3 m] of BF16 parts (K: the row's hi word split into three
// BF16 parts per coordinate; columns: the vertex's FP32 coordinates split likewise), FP32
// accumulators in TMEM, then a certified sign test per (row, vertex) with FP64 close calls on
// the exact pair; the 6 box rows on the ALU.  status[i] = 0 when every row holds at every vertex,
// 1 when a row is violated or within the tolerance band (the block kernel then solves the cell).
struct CheckArgs {
    const CheckRec *rec;
    const unsigned long long *count;  // records (read on the device)
    const float *rows;
    int64_t begin;
    int N;
    float box, box_lo;
    double delta;
    int *status;
    unsigned long long *counters;     // close calls are added to counters[kCloseCalls]
    int *err;                         // set to 1 when a pipeline wait timed out
};
cudaError_t prepare_check_tc();
void launch_check_tc(const CheckArgs &a, int sms, cudaStream_t st);
int march_smem_bytes(int max_n, int max_w);
int proposal_max_hidden();      // widest proposal hidden layer the march can evaluate
cudaError_t prepare_march_kernels(int max_n, int max_w, int *blocks_per_sm);
// mode 0 = FP64, 1 = double-float (mixed); persistent = ticket queue, else one level [begin, end)
void launch_march(const MarchArgs &a, int mode, bool persistent, int grid, cudaStream_t st);
// compose only: rows (n x (N + 1) x 4 doubles, a_F last) and errors of the cells with the given
// keys (n x key_words words) of one net; mode as launch_march (a.tc selects the tensor cores)
void launch_compose(const MarchArgs &a, int mode, const NetDev *net, const unsigned long long *keys, int key_words,
                    int64_t n, double *rows, float *err, cudaStream_t st);
// whether the tensor-core compose's scratch fits a net (width[1..L]) in a context of max_n rows
bool tc_fits(const int *width, int L, int max_n);

struct SeedArgs {
    const NetDev *nets;
    Arena ar;
    int net;
    int n_rays;
    const double *origins, *dirs;   // device, n_rays x 3
    double R;
    int max_halvings;
    int max_n, max_w;
    unsigned long long *seed_keys;  // device, n_rays x kw
    double *seed_x;                 // device, n_rays x 3
    int *seed_ok;                   // device, n_rays: 1 ok, -4 no sign change, -5 no common cell
    unsigned long long *n_new;      // device counter of new live seed cells
    int df;                         // 1: the double-float dichotomy (nets without hidden shortcuts,
                                    // pooling or leaky units), 0: FP64
};
cudaError_t prepare_seed_kernels(int max_n, int max_w);
void launch_seed(const SeedArgs &a, cudaStream_t st);

// sphere tracing (Sec. 4.3.1): one block per start point; writes the bracket segment of each
// start (origin, direction; t in [0, 1]) for launch_seed
struct TraceArgs {
    const NetDev *nets;
    int net;
    int n;                          // start points
    const double *starts;           // device, n x 3
    double eta, eps, pad;
    int max_steps;
    int max_n, max_w;
    double *origins, *dirs;         // device, n x 3 each (outputs)
};
void launch_trace(const TraceArgs &a, cudaStream_t st);

// random-pair sampling (Sec. 4.3.2): F at every sample, then segment r from the r-th negative
// sample to the r-th positive one, r < min(#neg, #pos, max_pairs)
struct PairArgs {
    const NetDev *nets;
    int net;
    int n_points, max_pairs;
    const double *points;           // device, n_points x 3
    double *F;                      // device, n_points (scratch)
    int *neg_idx, *pos_idx;         // device, max_pairs each (scratch)
    int max_n, max_w;
    double *origins, *dirs;         // device, max_pairs x 3 each (outputs)
    int *n_pairs;                   // device, 1 (output)
    int df;                         // 1: F in double-float (as SeedArgs.df), 0: FP64
};
void launch_pairs(const PairArgs &a, cudaStream_t st);

// ---- learned proposal on the tensor cores: one batch of cells per call (am_prop_tc.cu)
struct PropTC {
    bool ok = false;                    // shape supported (n_in <= 64, hidden in 64..256 step 64, n_out % 16)
    int n_in = 0, hidden = 0, n_out = 0, max_rows = 0;
    __nv_bfloat16 *X = nullptr;         // max_rows x 64 (features, zero padded)
    __nv_bfloat16 *H1 = nullptr, *H2 = nullptr;   // max_rows x hidden
    __nv_bfloat16 *W1p = nullptr;       // hidden x 64 (W1 zero padded)
    __nv_bfloat16 *scores = nullptr;    // max_rows x n_out (the march's scores)
    int *err = nullptr;                 // set to 1 by a CTA whose pipeline wait timed out
    alignas(64) unsigned char maps[6][128];   // TMA descriptors: X, H1, H2, W1p, W2, W3
};
// features of the cells [c0, c0 + n) of a level batch, as the in-march proposal computes them
struct PropFeatures {
    const unsigned long long *keys;     // arena keys (cell id stride kw)
    int kw;
    const float *entry_pt;              // arena entry points (3 per cell id)
    int64_t c0, n;
    const float *rows;                  // the batch's composed rows, FP32 pairs, a_F at row N
    int64_t rstride;                    // floats per cell ((N + 1) x 8)
    int N, L;
    int row0[kMaxLayers + 1], width[kMaxLayers + 1];
    __nv_bfloat16 *X;                   // set by prop_tc_features
};
bool prop_tc_shape_ok(int n_in, int hidden, int n_out);
cudaError_t prop_tc_alloc(PropTC &t, int n_in, int hidden, int n_out, int max_rows, const __nv_bfloat16 *W2,
                          const __nv_bfloat16 *W3);
void prop_tc_free(PropTC &t);
// room for at least rows cells in the activation and score buffers (the tensor maps over them are
// encoded again; the weights and their maps are kept)
cudaError_t prop_tc_grow(PropTC &t, int rows);
void prop_tc_sync_weights(PropTC &t, const float *W1, cudaStream_t st);
cudaError_t prop_tc_pack(const PropTC &t, const float *X, int rows, cudaStream_t st);
cudaError_t prop_tc_features(const PropTC &t, const PropFeatures &f, cudaStream_t st);
// the three layers for rows <= max_rows cells whose features are in t.X; the scores (rows x
// n_out) to out (ldo elements per row), FP32 or BF16
cudaError_t prop_tc_forward(const PropTC &t, const float *b1, const float *b2, const float *b3, int rows, void *out,
                            bool out_f32, int ldo, int *err, cudaStream_t st);

// ---- learned proposal (training and batch inference)
struct ProposalDev {
    int n_in = 0, hidden = 0, n_out = 0, max_batch = 0;
    int64_t off[7] = {};
    int64_t n_params = 0;
    int64_t step = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // FP32 master weights, grads, Adam state
    __nv_bfloat16 *wb = nullptr, *w2t = nullptr, *w3t = nullptr;     // BF16 copies
    float *buf[8] = {};
    __nv_bfloat16 *bbuf[4] = {};
    float *loss_parts = nullptr;
    PropTC tc;                     // forward pass on the tensor cores (when the shape allows)
};
cudaError_t proposal_alloc(ProposalDev &p, int n_in, int hidden, int n_out, int max_batch);
void proposal_free(ProposalDev &p);
void proposal_sync_copies(ProposalDev &p, cudaStream_t st);
cudaError_t proposal_forward(ProposalDev &p, const float *X, int n, float *Z, cudaStream_t st);
cudaError_t proposal_grad(ProposalDev &p, const float *X, const float *Y, int n, float *loss, cudaStream_t st);
cudaError_t proposal_train(ProposalDev &p, const float *X, const float *Y, int64_t n, int batch, int steps, float lr,
                           float *losses, cudaStream_t st);

// ---- mesh assembly
struct AsmArgs {
    Arena ar;
    const NetDev *nets;
    int64_t n_cells;
    int n_nets;
    unsigned long long *face_count;   // n_nets
    unsigned long long *face_fill;    // n_nets
    unsigned long long *face_base;    // n_nets (exclusive scan of face_count)
    unsigned long long *vert_count;   // n_nets
    unsigned long long *vert_base;    // n_nets
    int32_t *perm;                    // faces, grouped by net: cell ids
    int64_t *corner_off;              // faces + 1
    int32_t *corner_vid;              // corners: vertex id local to the net
    unsigned long long *vslots;       // vertex hash table
    unsigned long long vslot_mask;
    double *out_xyz;                  // 3 x vertices
    int32_t *out_fv;                  // corners
    int32_t *out_edges;               // corners
    unsigned long long *out_keys;     // faces x kw
    int64_t n_faces;
};
// Training samples of the learned proposal from an assembled mesh: one per corner of every face
// of one net (faces f0 .. f0 + nf - 1 of the assembled order, corners from c0), truncated at
// max_samples.  X: samples x n_in FP32, Y: samples x N FP32 (0/1 edge-neuron labels).
struct SampleArgs {
    Arena ar;
    const int32_t *perm;
    const int64_t *coff;
    int64_t f0, nf, c0, max_samples;
    int N, L, n_in;
    int row0[kMaxLayers + 2];
    int width[kMaxLayers + 1];
    float *X, *Y;
};
void launch_proposal_samples(const SampleArgs &a, cudaStream_t st);

void launch_asm_count(const AsmArgs &a, cudaStream_t st);
void launch_asm_scatter(const AsmArgs &a, cudaStream_t st);
cudaError_t launch_asm_offsets(const AsmArgs &a, int64_t *scan_tmp, int64_t scan_tmp_len, cudaStream_t st);
void launch_asm_vertices(const AsmArgs &a, cudaStream_t st);
void launch_asm_lookup(const AsmArgs &a, cudaStream_t st);
void launch_asm_write(const AsmArgs &a, cudaStream_t st);
// out[i] = in[i] - base, i < n (one net's face offsets from the context's global corner offsets)
void launch_rebase_offsets(const int64_t *in, int64_t base, int64_t *out, int64_t n, cudaStream_t st);

// ---- compose on the tcgen05 tensor cores with error-free BF16 digit planes (am_tc.cu)
constexpr int kOzDigits = 8;          // digit planes per operand (and accumulator diagonals)
constexpr int kOzBeta = 6;            // bits per digit
constexpr int kOzMaxFanIn = 1638;     // n_{l-1} * (largest diagonal's digit products) < 2^24
// one net as the sliced compose reads it (host struct holding device pointers)
struct OzNet {
    int L = 0, N = 0;
    int width[kMaxLayers + 1] = {}, row0[kMaxLayers + 1] = {};
    const double *Cl[kMaxLayers + 1] = {};
    const float *Clhi[kMaxLayers + 1] = {}, *Cllo[kMaxLayers + 1] = {};   // C_l as double-float pairs
    const int *eA[kMaxLayers + 1] = {};       // row exponents of W_l (device)
    const void *mapA[kMaxLayers + 1] = {};    // host CUtensorMap over the digit planes of W_l
    const double *AT[kMaxLayers + 1] = {};    // hidden part of W_l transposed (n_{l-1} x n_l), FP64
    const double *w_out = nullptr;
    double b_out = 0.0;
};
struct OzScratch {
    __nv_bfloat16 *B = nullptr;   // kOzDigits x 4 batch_cells x Kp digit planes of the stacked operand
    int *eB[2] = {nullptr, nullptr};   // 4 batch_cells column exponents, for alternate layers
    long long *P = nullptr;       // 4 batch_cells x Mp exact products of one layer (64-bit integers) ...
    long long *Q = nullptr;       // ... and the raw sums of its last diagonal, rounded once by the prep
    int *err = nullptr;           // set to 1 by a kernel whose pipeline wait timed out
    int64_t batch_cells = 0;      // multiple of 16
    int64_t *issued = nullptr;    // host counter: BF16 multiply-adds issued on the tensor cores
    int64_t *dirty = nullptr;     // host: P and Q may be non-zero in their first *dirty elements (a split-K
                                  // product needs zeros; the prep of a split product zeroes what it reads)
};
int oz_kp(int width);             // K padded to the 64-element staging chunk
int oz_mp(int width);             // rows padded to the 128-row tile
const int *oz_tile_cells(int *n); // the supported cells per CTA (UMMA N = 4 x cells); 0 = automatic per batch
void oz_slice_weights(const double *W, int n, int np, int fan, std::vector<uint16_t> &planes, std::vector<int> &eA);
cudaError_t oz_encode_weights(void *map, const void *planes, int n, int np);
int64_t oz_scratch_elems(int64_t batch_cells, int max_kp);

// ---- rank-1 neighbour compose (sliced level march).  A cell entered across neuron k of layer l
// has its parent's rows with row k's sign flipped (Z_1..Z_l are unchanged, s_k flips), and for
// j > l Z_j changes by the rank-1 term v_j a~^T: a~ = delta Z_l[k] (delta = +1 if k turns active,
// -1 if it turns inactive), v_{l+1} = W_{l+1}[:, k], v_j = W_j diag(s_{j-1}) v_{j-1}; a_F by
// (w_out . diag(s_L) v_L) a~ (w_out[k] a~ when l = L).  One operand column per cell.
struct R1Rows {
    int row0[kMaxLayers + 2];         // first neuron of each layer, row0[L + 1] = N
};
struct R1Scratch {
    int32_t *full_list = nullptr;     // cells of the level composed in full
    int32_t *r1_list = nullptr;       // cells composed by the rank-1 update, grouped by flip layer (ascending)
    int64_t list_cap = 0;
    int *it_l = nullptr;              // per item of a rank-1 batch: flip layer, flip index within it
    int *it_k = nullptr;
    float *it_a = nullptr;            // per item: a~ as FP32 pairs, [hi x 4 | lo x 4]
    int64_t item_cap = 0;
    unsigned long long *counts = nullptr;   // device: [0] full, [l] rank-1 with flip layer l
    int *offs = nullptr;              // device: [l] first r1_list slot of flip layer l, [kMaxLayers + 1 + l] cursors
};
// classify the cells [c_begin, n) of the next level (n = the cell counter, read on the device):
// rank-1 when the parent lies in [p0, p1) (the level just solved) and its chain is below max_chain
cudaError_t oz_rank1_classify(const OzNet &net, const Arena &ar, int64_t p0, int64_t p1, int64_t c_begin,
                              int max_chain, R1Scratch &r, cudaStream_t st);
// scatter the cells [c0, c1) into r.full_list and r.r1_list (offsets of the flip layers given)
cudaError_t oz_rank1_scatter(const Arena &ar, int64_t c0, int64_t c1, const int *h_offs, int L, R1Scratch &r,
                             cudaStream_t st);
// rows of the n cells r1_list[0..n) (sorted by flip layer; cnt_le[l] = how many have flip layer
// <= l) from their parents' rows (prev_rows, cell c at (c - prev0) (N + 1) x 32 B) into rows
// (cell c at (c - cell0) ...), FP32 pairs
struct R1Cells {
    const unsigned long long *keys;   // cell c's key at keys + c kw (the child's key)
    int kw;
    const int32_t *parent;            // cell c's parent: its rows at prev_rows + (parent[c] - prev0) ...
    const int32_t *entry;             // the flipped neuron of cell c
};
cudaError_t oz_rank1(const OzNet &net, const R1Cells &cells, const int32_t *list, int64_t n, const int64_t *cnt_le,
                     const void *prev_rows, int64_t prev0, void *rows, int64_t cell0, const OzScratch &scr,
                     R1Scratch &r, int tile_cells, int sms, cudaStream_t st);
// FP64 rows (n cells x (N + 1) rows x 4 doubles) <-> FP32 pairs (per cell: the N + 1 hi words
// [hi x 4], then the N + 1 lo words [lo x 4]); rows_per_cell = N + 1
void rows_to_pairs(const double *rows, float *pairs, int64_t n_cells, int rows_per_cell, cudaStream_t st);
void pairs_to_rows(const float *pairs, double *rows, int64_t n_cells, int rows_per_cell, cudaStream_t st);
// rows of the cells with keys (n x kw words): n x (N + 1) rows of 32 bytes, a_F last, each row
// FP64 [a | a0] or, with df, FP32 pairs (the N + 1 hi words [hi x 4], then the N + 1 lo words
// [lo x 4]); batches smaller than sms x the tiles
// resident per SM split the product's K over several CTAs; tile_cells 0 picks the tile per batch
// list (optional): the batch is the cells list[0..n) (keys at keys + list[i] kw, rows at rows +
// (list[i] - cell0) x (N + 1) x 32 B)
cudaError_t oz_compose(const OzNet &net, const unsigned long long *keys, int kw, int64_t n, void *rows, bool df,
                       const OzScratch &scr, int tile_cells, int sms, cudaStream_t st, const int32_t *list = nullptr,
                       int64_t cell0 = 0);

}  // namespace am
