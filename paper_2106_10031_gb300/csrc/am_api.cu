// am_api.cu -- host side of the C ABI (include/analytic_marching.h).
//
// The context owns every device buffer, allocated once at creation (the cell arena, the
// hash table, the net weights) or grown on demand (mesh assembly).  am_march runs
// Algorithm 1 breadth first: one launch of the cell kernel per level over the id range of
// that level's active cells, until a level pushes no new cell; then the assembly kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/analytic_marching.h"
#include "am_kernels.h"

using namespace am;

namespace {

constexpr int kMaxNets = 1024;
constexpr int kMaxTriggerPoints = 1 << 24;   // start points / samples per trigger call
constexpr int kMaxTraceSteps = 1 << 16;      // sphere-tracing step budget
constexpr double kTracePad = 1e-9;           // half-length pad of the bracket after tracing
constexpr unsigned long long kZobristSeed = 0x2106100310031ull;
constexpr long long kWaitNs = 4000000000ll;  // 4 s limit on any wait for work in the persistent march

struct NetHost {
    NetDev dev;              // device pointers into `blob`, `fblob` and `tblob`
    double *blob = nullptr;  // device allocation holding AT, Cl, w_out (FP64)
    float *fblob = nullptr;  // the same as double-float pairs (hi, lo)
    void *tblob = nullptr;   // BF16 hi/lo fragments of W_l and row norms (tensor-core compose)
    void *ozblob = nullptr;  // BF16 digit planes of W_l and their row exponents (sliced compose)
    struct alignas(64) MapBytes { unsigned char b[128]; };
    std::vector<MapBytes> ozmap;     // TMA descriptor over each layer's digit planes (index l)
    size_t oz_off_eA[kMaxLayers + 1] = {};
    bool oz_ok = false;      // every hidden fan-in fits the exact accumulation
    int N = 0, max_w = 0;
};

// FP32 -> BF16, round to nearest even (finite inputs)
uint16_t bf16_rn(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float bf16_to_float(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

struct MeshInfo {
    int64_t faces = 0, face_base = 0, corners = 0, corner_base = 0, verts = 0, vert_base = 0, open = 0;
};

}  // namespace

struct am_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    am_ctx_opts opts{};
    Arena ar{};
    NetDev *d_nets = nullptr;
    std::vector<NetHost> nets;
    int max_n_loaded = 1, max_w_loaded = 1;
    int sm_count = 0, blocks_per_sm = 0;
    int64_t solved_upto = 0;       // cells [0, solved_upto) are solved
    am_stats_t stats{};
    std::string err;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, evk0 = nullptr, evk1 = nullptr;
    std::vector<cudaEvent_t> oz_ev;    // sliced march: 3 events per batch of a level, read after the level
    int oz_err_host = 0;               // sliced march: the pipeline time-out flag, copied with the counters
    int64_t oz_dirty = 0;              // sliced compose: leading elements of P and Q that may be non-zero
    // seeding scratch (grown on demand)
    double *d_rays = nullptr;
    unsigned long long *d_seed_keys = nullptr;
    double *d_seed_x = nullptr;
    int *d_seed_ok = nullptr;
    int seed_cap = 0;
    // assembly buffers (grown on demand)
    unsigned long long *d_netcnt = nullptr;   // 5 x kMaxNets
    int32_t *d_perm = nullptr;
    int64_t *d_coff = nullptr;
    int64_t coff_cap = 0;
    int64_t *d_coff_net = nullptr;     // am_get_mesh_device: each net's face offsets rebased to 0
    int64_t coff_net_cap = 0;
    double *d_trig = nullptr;          // trigger samples / start points and their scratch
    int64_t trig_cap = 0;
    int64_t *d_scan_tmp = nullptr;
    int64_t scan_tmp_len = 0;
    int64_t faces_cap = 0;
    int32_t *d_cvid = nullptr, *d_fv = nullptr, *d_fe = nullptr;
    int64_t corners_cap = 0;
    double *d_xyz = nullptr;
    int64_t verts_cap = 0;
    unsigned long long *d_fkeys = nullptr;
    int64_t fkeys_cap = 0;
    unsigned long long *d_vslots = nullptr;
    int64_t vslots_n = 0;
    std::vector<MeshInfo> mesh;
    bool mesh_valid = false;
    ProposalDev prop;
    OzScratch oz;                 // sliced tensor-core compose (allocated on first use)
    int oz_tile_cells = 0;        // cells per tensor-core tile (0 = default 16)
    int oz_rank1_period = 0;      // rank-1 compose: full compose every this many generations (0 = 32)
    int clip_kernel = 0;          // sliced march: 0 warp-per-cell clip with block fallback, 1 block kernel
    int check_kernel = 0;         // sliced march, warp clip: 0 check in the warp, 1 dense check on the tensor cores
    int32_t *fb_list = nullptr;   // the warp clip's fallback cells (one level) and their count
    unsigned long long *fb_count = nullptr;
    unsigned long long *clip_work = nullptr;   // the warp clip's cell counter (zeroed before each launch)
    CheckRec *chk = nullptr;      // the tensor-core check's records (one chunk), their count and status
    unsigned long long *chk_count = nullptr;
    int *chk_status = nullptr;
    // march with AM_PREC_SLICED: the rows of the level being solved and of the level before it
    // (the parents of the next level's rank-1 composes), FP32 pairs, (N + 1) x 32 B per cell
    double *lv_rows[2] = {nullptr, nullptr};
    int64_t lv_cap[2] = {0, 0};   // cells
    R1Scratch r1;
    unsigned long long r1_hcounts[kMaxLayers + 1] = {};
    bool r1_planned = false;      // the cells of the next level are classified (r1_hcounts valid)
    int64_t r1_prev0 = 0;         // first cell of the level whose rows the other buffer holds
    // time-out path: the next persistent march hands out test_stall_ids ids it never publishes
    // and waits at most test_wait_ns for work (am_test_stall_next_march); after a time-out the
    // context marches again only after am_reset
    int64_t test_stall_ids = 0;
    long long test_wait_ns = 0;
    bool timed_out = false;
};

namespace {

am_status fail(am_ctx *c, am_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define CU(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(ctx, AM_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                        __FILE__, __LINE__);                                                          \
    } while (0)

int64_t pow2_at_least(int64_t x)
{
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

template <class T>
cudaError_t grow(T **p, int64_t *cap, int64_t need)
{
    if (need <= *cap && *p) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    int64_t n = std::max<int64_t>(need, 1024);
    n = n + n / 4;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * n);
    *cap = e == cudaSuccess ? n : 0;
    return e;
}

am_status sync_status(am_ctx *ctx, unsigned long long *host_counters)
{
    CU(cudaMemcpyAsync(host_counters, ctx->ar.counters, sizeof(unsigned long long) * kNumCounters,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return AM_OK;
}

am_status status_error(am_ctx *ctx, unsigned long long st)
{
    if (st & kStCellCap) return fail(ctx, AM_ERR_CAPACITY, "cell capacity (max_cells=%lld) exceeded",
                                     (long long)ctx->ar.cap);
    if (st & kStHashFull) return fail(ctx, AM_ERR_CAPACITY, "cell hash table probe limit reached");
    if (st & kStFaceVerts) return fail(ctx, AM_ERR_CAPACITY, "a face has more than max_face_verts=%d corners",
                                       ctx->ar.maxv);
    if (st & kStVertHash) return fail(ctx, AM_ERR_CAPACITY, "vertex hash table probe limit reached");
    if (st & kStTimeout) return fail(ctx, AM_ERR_TIMEOUT, "a bounded device wait gave up");
    return AM_OK;
}

// Scratch of the sliced compose: digit planes of a batch of cells, their column exponents and
// the pipeline time-out flag; sized for the widest loadable layer.
am_status ensure_oz_scratch(am_ctx *ctx)
{
    if (ctx->oz.B) return AM_OK;
    OzScratch &z = ctx->oz;
    z.batch_cells = 4096;
    z.issued = &ctx->stats.tensor_macs;
    z.dirty = &ctx->oz_dirty;
    CU(cudaMalloc(&z.B, sizeof(__nv_bfloat16) * oz_scratch_elems(z.batch_cells, oz_kp(ctx->opts.max_width))));
    CU(cudaMalloc(&z.eB[0], sizeof(int) * 4 * z.batch_cells));
    CU(cudaMalloc(&z.eB[1], sizeof(int) * 4 * z.batch_cells));
    CU(cudaMalloc(&z.P, sizeof(long long) * 4 * z.batch_cells * oz_mp(ctx->opts.max_width)));
    CU(cudaMalloc(&z.Q, sizeof(long long) * 4 * z.batch_cells * oz_mp(ctx->opts.max_width)));
    CU(cudaMalloc(&z.err, sizeof(int)));
    CU(cudaMemsetAsync(z.err, 0, sizeof(int), ctx->stream));
    // the products start at zero; every kernel that reads a product zeroes it again
    CU(cudaMemsetAsync(z.P, 0, sizeof(long long) * 4 * z.batch_cells * oz_mp(ctx->opts.max_width), ctx->stream));
    CU(cudaMemsetAsync(z.Q, 0, sizeof(long long) * 4 * z.batch_cells * oz_mp(ctx->opts.max_width), ctx->stream));
    return AM_OK;
}

OzNet oz_view(const NetHost &nh)
{
    OzNet v;
    const NetDev &d = nh.dev;
    v.L = d.L;
    v.N = d.N;
    for (int l = 1; l <= d.L; ++l) {
        v.width[l] = d.width[l];
        v.row0[l] = d.row0[l];
        v.Cl[l] = d.Cl[l];
        v.Clhi[l] = d.Clhi[l];
        v.Cllo[l] = d.Cllo[l];
        v.AT[l] = d.AT[l];
        if (l >= 2) {
            v.eA[l] = reinterpret_cast<const int *>(reinterpret_cast<const unsigned char *>(nh.ozblob) + nh.oz_off_eA[l]);
            v.mapA[l] = nh.ozmap[l].b;
        }
    }
    v.w_out = d.w_out;
    v.b_out = d.b_out;
    return v;
}

// rows (n x (N + 1) x 4) of n cells of one net on the tensor cores, asynchronous on the stream
// d_keys: cell i's key at d_keys + i * key_stride words (the net's own width for am_compose's
// caller-packed keys, the arena's width inside the march)
am_status sliced_compose_async(am_ctx *ctx, int net_id, const unsigned long long *d_keys, int key_stride, int64_t n,
                               void *d_rows, bool df = false)
{
    const NetHost &nh = ctx->nets[net_id];
    if (!nh.oz_ok)
        return fail(ctx, AM_ERR_INVALID_ARG, "AM_PREC_SLICED needs every hidden fan-in <= %d", kOzMaxFanIn);
    am_status s = ensure_oz_scratch(ctx);
    if (s != AM_OK) return s;
    const int tile = ctx->oz_tile_cells;                   // 0: automatic per batch
    CU(oz_compose(oz_view(nh), d_keys, key_stride, n, d_rows, df, ctx->oz, tile, ctx->sm_count, ctx->stream));
    const int64_t batches = (n + ctx->oz.batch_cells - 1) / ctx->oz.batch_cells;
    ctx->stats.kernel_launches += (2 * (int64_t)nh.dev.L - 1) * batches;
    return AM_OK;
}

// AM_ERR_TIMEOUT if a tensor-core pipeline wait gave up since the last check (synchronises)
am_status sliced_check(am_ctx *ctx)
{
    int herr = 0;
    CU(cudaMemcpyAsync(&herr, ctx->oz.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (herr) {
        CU(cudaMemsetAsync(ctx->oz.err, 0, sizeof(int), ctx->stream));
        // an aborted product may have left partial sums unread: start from zero again
        const size_t pq = sizeof(long long) * 4 * ctx->oz.batch_cells * oz_mp(ctx->opts.max_width);
        CU(cudaMemsetAsync(ctx->oz.P, 0, pq, ctx->stream));
        CU(cudaMemsetAsync(ctx->oz.Q, 0, pq, ctx->stream));
        ctx->oz_dirty = 0;
        return fail(ctx, AM_ERR_TIMEOUT, "a tensor-core pipeline wait of the sliced compose gave up");
    }
    return AM_OK;
}

am_status sliced_compose(am_ctx *ctx, int net_id, const unsigned long long *d_keys, int64_t n, double *d_rows)
{
    am_status s = sliced_compose_async(ctx, net_id, d_keys, ctx->nets[net_id].dev.kw, n, d_rows);
    return s != AM_OK ? s : sliced_check(ctx);
}

}  // namespace

extern "C" {

am_status am_create(am_ctx **out, const am_ctx_opts *o)
{
    am_ctx *ctx = nullptr;
    if (!out) return AM_ERR_INVALID_ARG;
    *out = nullptr;
    ctx = new am_ctx();
    am_ctx_opts d{};
    if (o) d = *o;
    if (d.max_cells <= 0) d.max_cells = 1 << 20;
    if (d.max_face_verts <= 0) d.max_face_verts = 32;
    if (d.max_neurons <= 0) d.max_neurons = 4096;
    if (d.max_width <= 0) d.max_width = 512;
    if (d.max_cells > kMaxCellIds || d.max_face_verts < 8 || d.max_face_verts > 62 || d.max_neurons > kMaxNeurons) {
        am_status s = fail(ctx, AM_ERR_INVALID_ARG, "capacity out of range");
        *out = ctx;
        return s;
    }
    d.hash_slots = pow2_at_least(std::max<int64_t>(d.hash_slots, 2 * d.max_cells));
    ctx->opts = d;
    ctx->device = d.device;
    *out = ctx;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= d.device || d.device < 0)
        return fail(ctx, AM_ERR_CUDA, "no usable CUDA device %d (count %d)", d.device, ndev);
    CU(cudaSetDevice(d.device));
    if (d.stream) {
        ctx->stream = (cudaStream_t)d.stream;
    } else {
        CU(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    CU(cudaEventCreate(&ctx->ev0));
    CU(cudaEventCreate(&ctx->ev1));
    CU(cudaEventCreate(&ctx->ev2));
    CU(cudaEventCreate(&ctx->evk0));
    CU(cudaEventCreate(&ctx->evk1));
    Arena &ar = ctx->ar;
    ar.kw = (d.max_neurons + 63) / 64;
    ar.maxv = d.max_face_verts;
    ar.cap = d.max_cells;
    ar.slot_mask = (unsigned long long)(d.hash_slots - 1);
    CU(cudaMalloc(&ar.keys, sizeof(unsigned long long) * ar.kw * ar.cap));
    CU(cudaMalloc(&ar.net, sizeof(int32_t) * ar.cap));
    CU(cudaMalloc(&ar.hash, sizeof(unsigned long long) * ar.cap));
    CU(cudaMalloc(&ar.nverts, sizeof(int32_t) * ar.cap));
    CU(cudaMalloc(&ar.edges, sizeof(int32_t) * ar.cap * ar.maxv));
    CU(cudaMalloc(&ar.verts, sizeof(double) * 3 * ar.cap * ar.maxv));
    CU(cudaMalloc(&ar.ready, sizeof(unsigned) * ar.cap));
    CU(cudaMalloc(&ar.entry_plane, sizeof(int32_t) * ar.cap));
    CU(cudaMalloc(&ar.entry_pt, sizeof(float) * 3 * ar.cap));
    CU(cudaMalloc(&ar.parent, sizeof(int32_t) * ar.cap));
    CU(cudaMalloc(&ar.chain, sizeof(int32_t) * ar.cap));
    CU(cudaMalloc(&ar.cls, sizeof(int32_t) * ar.cap));
    CU(cudaMalloc(&ar.slots, sizeof(unsigned long long) * d.hash_slots));
    CU(cudaMalloc(&ar.counters, sizeof(unsigned long long) * kNumCounters));
    {
        std::vector<unsigned long long> z(64 * ar.kw);
        for (size_t k = 0; k < z.size(); ++k) z[k] = splitmix64(kZobristSeed + 0x632BE59BD9B4E019ull * (k + 1));
        unsigned long long *dz = nullptr;
        CU(cudaMalloc(&dz, sizeof(unsigned long long) * z.size()));
        CU(cudaMemcpy(dz, z.data(), sizeof(unsigned long long) * z.size(), cudaMemcpyHostToDevice));
        ar.zob = dz;
    }
    CU(cudaMalloc(&ctx->d_nets, sizeof(NetDev) * kMaxNets));
    CU(cudaMalloc(&ctx->d_netcnt, sizeof(unsigned long long) * 6 * kMaxNets));
    CU(cudaMemsetAsync(ar.slots, 0, sizeof(unsigned long long) * d.hash_slots, ctx->stream));
    CU(cudaMemsetAsync(ar.counters, 0, sizeof(unsigned long long) * kNumCounters, ctx->stream));
    CU(cudaMemsetAsync(ar.ready, 0, sizeof(unsigned) * ar.cap, ctx->stream));
    {
        const int smem = march_smem_bytes(d.max_neurons, d.max_width);
        int optin = 0;
        CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d.device));
        if (smem > optin)
            return fail(ctx, AM_ERR_INVALID_ARG, "max_neurons=%d / max_width=%d need %d B of shared memory per block "
                        "(device allows %d)", d.max_neurons, d.max_width, smem, optin);
    }
    CU(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, d.device));
    CU(prepare_march_kernels(d.max_neurons, d.max_width, &ctx->blocks_per_sm));
    if (ctx->blocks_per_sm < 1) return fail(ctx, AM_ERR_CUDA, "the march kernel cannot be resident");
    CU(prepare_seed_kernels(d.max_neurons, d.max_width));
    CU(prepare_clip_warp());
    CU(prepare_check_tc());
    CU(cudaStreamSynchronize(ctx->stream));
    return AM_OK;
}

void am_destroy(am_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream) {
        cudaSetDevice(ctx->device);
        cudaStreamSynchronize(ctx->stream);
    }
    Arena &ar = ctx->ar;
    void *bufs[] = {ar.keys, ar.net, ar.hash, ar.nverts, ar.edges, ar.verts, ar.slots, ar.counters,
                    ar.ready, ar.entry_plane, ar.entry_pt, ar.parent, ar.chain, ar.cls,
                    (void *)ar.zob, ctx->d_nets, ctx->d_netcnt, ctx->d_rays, ctx->d_seed_keys, ctx->d_seed_x,
                    ctx->d_seed_ok, ctx->d_perm, ctx->d_coff, ctx->d_coff_net, ctx->d_trig, ctx->d_scan_tmp, ctx->d_cvid, ctx->d_fv,
                    ctx->d_fe,
                    ctx->d_xyz, ctx->d_fkeys, ctx->d_vslots};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (auto &n : ctx->nets) {
        if (n.blob) cudaFree(n.blob);
        if (n.fblob) cudaFree(n.fblob);
        if (n.tblob) cudaFree(n.tblob);
        if (n.ozblob) cudaFree(n.ozblob);
    }
    if (ctx->oz.B) cudaFree(ctx->oz.B);
    for (void *b : {(void *)ctx->oz.eB[0], (void *)ctx->oz.eB[1], (void *)ctx->oz.P, (void *)ctx->oz.Q})
        if (b) cudaFree(b);
    if (ctx->oz.err) cudaFree(ctx->oz.err);
    for (int b = 0; b < 2; ++b)
        if (ctx->lv_rows[b]) cudaFree(ctx->lv_rows[b]);
    if (ctx->fb_list) cudaFree(ctx->fb_list);
    if (ctx->fb_count) cudaFree(ctx->fb_count);
    if (ctx->clip_work) cudaFree(ctx->clip_work);
    if (ctx->chk) cudaFree(ctx->chk);
    if (ctx->chk_count) cudaFree(ctx->chk_count);
    if (ctx->chk_status) cudaFree(ctx->chk_status);
    for (void *b : {(void *)ctx->r1.full_list, (void *)ctx->r1.r1_list, (void *)ctx->r1.it_l, (void *)ctx->r1.it_k,
                    (void *)ctx->r1.it_a, (void *)ctx->r1.counts, (void *)ctx->r1.offs})
        if (b) cudaFree(b);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->ev2) cudaEventDestroy(ctx->ev2);
    if (ctx->evk0) cudaEventDestroy(ctx->evk0);
    if (ctx->evk1) cudaEventDestroy(ctx->evk1);
    for (cudaEvent_t e : ctx->oz_ev)
        if (e) cudaEventDestroy(e);
    proposal_free(ctx->prop);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *am_last_error(const am_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

am_status am_load_mlp(am_ctx *ctx, const am_mlp_desc *dsc, int *net_id)
{
    if (!ctx || !dsc || !net_id) return fail(ctx, AM_ERR_INVALID_ARG, "null argument");
    if (!ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "context was not created successfully");
    const int L = dsc->n_hidden, zd = dsc->latent_dim, in_dim = 3 + zd;
    if (L < 1 || L > kMaxLayers || zd < 0 || (zd > 0 && !dsc->latent) || !dsc->width || !dsc->W || !dsc->b ||
        !dsc->w_out)
        return fail(ctx, AM_ERR_INVALID_ARG, "bad net description (layers %d, latent %d)", L, zd);
    if (dsc->skip_layer != 0 && (dsc->skip_layer < 2 || dsc->skip_layer > L))
        return fail(ctx, AM_ERR_INVALID_ARG, "skip_layer %d out of range", dsc->skip_layer);
    if (!(std::fabs(dsc->slope) < 1.0))
        return fail(ctx, AM_ERR_INVALID_ARG, "activation slope %g: |slope| < 1", dsc->slope);
    if ((int)ctx->nets.size() >= kMaxNets) return fail(ctx, AM_ERR_CAPACITY, "too many nets");
    int N = 0, mw = 0;
    for (int l = 0; l < L; ++l) {
        if (dsc->width[l] < 1 || !dsc->W[l] || !dsc->b[l]) return fail(ctx, AM_ERR_INVALID_ARG, "bad layer %d", l + 1);
        N += dsc->width[l];
        mw = std::max(mw, dsc->width[l]);
    }
    // final max pooling over M heads (Sec. 5.2): M pooling rows and key bits after the units
    const int M = dsc->n_heads >= 2 ? dsc->n_heads : 0;
    if (dsc->n_heads < 0 || dsc->n_heads > AM_MAX_HEADS || (M && (!dsc->w_heads || !dsc->b_heads)))
        return fail(ctx, AM_ERR_INVALID_ARG, "n_heads %d: 0, 1 or 2..%d with w_heads and b_heads", dsc->n_heads,
                    AM_MAX_HEADS);
    const int n_units = N;
    N += M;
    if (N > ctx->opts.max_neurons || mw > ctx->opts.max_width)
        return fail(ctx, AM_ERR_INVALID_ARG, "net has N=%d neurons, width %d; context allows %d, %d", N, mw,
                    ctx->opts.max_neurons, ctx->opts.max_width);
    // residual shortcuts (Sec. 5.1): S_l h_src added to layer l's pre-activation
    bool hidden_shortcut = false;
    if (dsc->shortcut_src) {
        for (int l = 1; l <= L; ++l) {
            const int src = dsc->shortcut_src[l - 1];
            if (src < 0) continue;
            if (src >= l)
                return fail(ctx, AM_ERR_INVALID_ARG, "layer %d: shortcut source %d is not an earlier layer", l, src);
            const int ns = src == 0 ? 3 : dsc->width[src - 1];
            const bool ident = !dsc->shortcut_S || !dsc->shortcut_S[l - 1];
            if (ident && ns != dsc->width[l - 1])
                return fail(ctx, AM_ERR_INVALID_ARG, "layer %d: an identity shortcut needs %d == %d units", l, ns,
                            dsc->width[l - 1]);
            hidden_shortcut = hidden_shortcut || src >= 1;
        }
    }
    auto sc_src = [&](int l) { return dsc->shortcut_src ? dsc->shortcut_src[l - 1] : -1; };
    auto sc_mat = [&](int l) -> const double * { return dsc->shortcut_S ? dsc->shortcut_S[l - 1] : nullptr; };
    // fold: Cl (n_l x 4) and AT (n_{l-1} x n_l), then w_out
    std::vector<double> host;
    std::vector<size_t> offC(L + 1), offA(L + 1);
    for (int l = 1; l <= L; ++l) {
        const int n = dsc->width[l - 1], np = l > 1 ? dsc->width[l - 2] : 0;
        const int fan = l == 1 ? in_dim : np + (l == dsc->skip_layer ? in_dim : 0);
        const double *W = dsc->W[l - 1], *b = dsc->b[l - 1];
        offC[l] = host.size();
        const int xoff = l == 1 ? 0 : (l == dsc->skip_layer ? np : -1);
        for (int k = 0; k < n; ++k) {
            double c[4] = {0.0, 0.0, 0.0, b[k]};
            if (xoff >= 0) {
                for (int i = 0; i < 3; ++i) c[i] = W[(size_t)k * fan + xoff + i];
                for (int j = 0; j < zd; ++j) c[3] += W[(size_t)k * fan + xoff + 3 + j] * dsc->latent[j];
            }
            if (sc_src(l) == 0) {                  // a shortcut from x: S_l x joins the constant rows
                const double *S = sc_mat(l);
                for (int i = 0; i < 3; ++i) c[i] += S ? S[(size_t)k * 3 + i] : (k == i ? 1.0 : 0.0);
            }
            host.insert(host.end(), c, c + 4);
        }
        offA[l] = host.size();
        if (l > 1) {
            host.resize(host.size() + (size_t)np * n);
            double *AT = host.data() + offA[l];
            for (int k = 0; k < n; ++k)
                for (int j = 0; j < np; ++j) AT[(size_t)j * n + k] = W[(size_t)k * fan + j];
        }
    }
    const size_t offW = host.size();
    host.insert(host.end(), dsc->w_out, dsc->w_out + dsc->width[L - 1]);
    const size_t offH = host.size();               // pooling heads: M x n_L weights, then M offsets
    if (M) {
        host.insert(host.end(), dsc->w_heads, dsc->w_heads + (size_t)M * dsc->width[L - 1]);
        host.insert(host.end(), dsc->b_heads, dsc->b_heads + M);
    }
    std::vector<size_t> offS(L + 1, 0);            // matrix shortcuts from hidden layers
    for (int l = 2; l <= L; ++l) {
        const int src = sc_src(l);
        if (src < 1 || !sc_mat(l)) continue;
        offS[l] = host.size();
        host.insert(host.end(), sc_mat(l), sc_mat(l) + (size_t)dsc->width[l - 1] * dsc->width[src - 1]);
    }
    // double-float split of every value: hi = fl32(x), lo = fl32(x - hi)
    std::vector<float> fhost(2 * host.size());
    for (size_t i = 0; i < host.size(); ++i) {
        const float h = (float)host[i];
        fhost[i] = h;
        fhost[host.size() + i] = (float)(host[i] - (double)h);
    }
    NetHost nh;
    CU(cudaMalloc(&nh.blob, sizeof(double) * host.size()));
    CU(cudaMalloc(&nh.fblob, sizeof(float) * fhost.size()));
    CU(cudaMemcpyAsync(nh.blob, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(nh.fblob, fhost.data(), sizeof(float) * fhost.size(), cudaMemcpyHostToDevice, ctx->stream));
    const size_t lo_off = host.size();
    NetDev &nd = nh.dev;
    memset(&nd, 0, sizeof nd);
    nd.L = L;
    nd.N = N;
    nd.kw = (N + 63) / 64;
    int r0 = 0;
    for (int l = 1; l <= L; ++l) {
        nd.width[l] = dsc->width[l - 1];
        nd.row0[l] = r0;
        r0 += nd.width[l];
        nd.Cl[l] = nh.blob + offC[l];
        nd.AT[l] = l > 1 ? nh.blob + offA[l] : nullptr;
        nd.Clhi[l] = nh.fblob + offC[l];
        nd.Cllo[l] = nh.fblob + lo_off + offC[l];
        nd.AThi[l] = l > 1 ? nh.fblob + offA[l] : nullptr;
        nd.ATlo[l] = l > 1 ? nh.fblob + lo_off + offA[l] : nullptr;
        nd.sc_src[l] = sc_src(l) >= 1 ? sc_src(l) : 0;
        nd.sc_S[l] = nd.sc_src[l] && offS[l] ? nh.blob + offS[l] : nullptr;
    }
    {
        // tensor-core operands: BF16 hi/lo of W_l (hidden part) in A-fragment order, row norms
        std::vector<size_t> offF(L + 1, 0), offN(L + 1, 0);
        size_t words = 0;                          // in uint4 units
        for (int l = 2; l <= L; ++l) {
            const int n = dsc->width[l - 1], np = dsc->width[l - 2];
            offF[l] = words;
            words += (size_t)((n + 15) / 16) * ((np + 15) / 16) * 96;
        }
        for (int l = 2; l <= L; ++l) {
            offN[l] = words;
            words += (size_t)(2 * dsc->width[l - 1] + 3) / 4;
        }
        std::vector<uint32_t> tb(4 * std::max<size_t>(words, 1), 0u);
        for (int l = 2; l <= L; ++l) {
            const int n = dsc->width[l - 1], np = dsc->width[l - 2];
            const int fan = np + (l == dsc->skip_layer ? in_dim : 0);
            const double *W = dsc->W[l - 1];
            const int Mt = (n + 15) / 16, Kt = (np + 15) / 16;
            auto wat = [&](int m, int k) { return (m < n && k < np) ? W[(size_t)m * fan + k] : 0.0; };
            for (int mt = 0; mt < Mt; ++mt)
                for (int kt = 0; kt < Kt; ++kt)
                    for (int lane = 0; lane < 32; ++lane) {
                        const int g = lane >> 2, t = lane & 3;
                        // a0..a7: (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1), then the same at k + 8
                        const int rows[8] = {g, g, g + 8, g + 8, g, g, g + 8, g + 8};
                        const int cols[8] = {2 * t, 2 * t + 1, 2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9, 2 * t + 8, 2 * t + 9};
                        uint16_t part[3][8];              // w = hi + mid + lo (+ |w| 2^-27)
                        for (int i = 0; i < 8; ++i) {
                            double w = wat(mt * 16 + rows[i], kt * 16 + cols[i]);
                            for (int q = 0; q < 3; ++q) {
                                part[q][i] = bf16_rn((float)w);
                                w -= (double)bf16_to_float(part[q][i]);
                            }
                        }
                        for (int q = 0; q < 3; ++q) {
                            uint32_t *t = tb.data() + 4 * (offF[l] + ((size_t)mt * Kt + kt) * 96 + 32 * q + lane);
                            for (int r = 0; r < 4; ++r)
                                t[r] = (uint32_t)part[q][2 * r] | ((uint32_t)part[q][2 * r + 1] << 16);
                        }
                    }
            float *wn = reinterpret_cast<float *>(tb.data() + 4 * offN[l]);     // (|W_m|_2, max_j |W_mj|)
            for (int m = 0; m < n; ++m) {
                double s2 = 0.0, mx = 0.0;
                for (int k = 0; k < np; ++k) {
                    const double w = W[(size_t)m * fan + k];
                    s2 += w * w;
                    mx = std::max(mx, fabs(w));
                }
                wn[2 * m] = (float)(sqrt(s2) * (1.0 + 1e-6));
                wn[2 * m + 1] = (float)(mx * (1.0 + 1e-6));
            }
        }
        CU(cudaMalloc(&nh.tblob, sizeof(uint32_t) * tb.size()));
        CU(cudaMemcpyAsync(nh.tblob, tb.data(), sizeof(uint32_t) * tb.size(), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));      // tb is released at the end of this scope
        for (int l = 2; l <= L; ++l) {
            nd.Wf[l] = reinterpret_cast<const uint4 *>(nh.tblob) + offF[l];
            nd.wn[l] = reinterpret_cast<const float *>(reinterpret_cast<const uint4 *>(nh.tblob) + offN[l]);
        }
    }
    nd.w_out = nh.blob + offW;
    nd.w_out_hi = nh.fblob + offW;
    nd.w_out_lo = nh.fblob + lo_off + offW;
    nd.b_out = dsc->b_out;
    nd.M = M;
    nd.n_units = n_units;
    nd.w_heads = M ? nh.blob + offH : nullptr;
    nd.b_heads = M ? nh.blob + offH + (size_t)M * dsc->width[L - 1] : nullptr;
    const int id = (int)ctx->nets.size();
    nd.salt = splitmix64(0xA11CE5EEDull + (unsigned long long)id * 0x9E3779B97F4A7C15ull);
    {
        // The mixed path's rigorous row-error bound grows layer by layer by at most the largest
        // row sum of |W_l| (hidden part); its per-product coefficient is 2 (n + 4)^2 u^2 with
        // u = 2^-24.  When the predicted relative bound at the last layer exceeds 1e-7, the
        // sign tests of this net cannot be certified in double-float and its cells go to FP64.
        double growth = 1.0, rel = 0.0;
        const double u = 5.9604644775390625e-8;
        for (int l = 1; l <= L; ++l) {
            const int n = dsc->width[l - 1], np = l > 1 ? dsc->width[l - 2] : 0;
            const int fan = l == 1 ? in_dim : np + (l == dsc->skip_layer ? in_dim : 0);
            if (l > 1) {
                double mx = 0.0;
                for (int k = 0; k < n; ++k) {
                    double rs = 0.0;
                    for (int j = 0; j < np; ++j) rs += fabs(dsc->W[l - 1][(size_t)k * fan + j]);
                    mx = std::max(mx, rs);
                }
                growth *= std::max(mx, 1.0);
            }
            rel += 2.0 * (np + 8.0) * (np + 8.0) * u * u * growth;
        }
        nd.df_ok = rel < 1e-7 && dsc->slope == 0.0 && !hidden_shortcut && !M ? 1 : 0;
    }
    nd.slope = dsc->slope;
    nd.fp64_only = dsc->slope != 0.0 || hidden_shortcut || M ? 1 : 0;
    {
        // sliced tensor-core compose: 8 BF16 digit planes of each hidden W_l, row exponents, and
        // a TMA descriptor per layer; only when every fan-in keeps the accumulation exact
        nh.oz_ok = !nd.fp64_only;               // the sliced operands mask with s_l alone, no shortcut
        for (int l = 2; l <= L; ++l) nh.oz_ok = nh.oz_ok && dsc->width[l - 2] <= kOzMaxFanIn;
        if (nh.oz_ok && L >= 2) {
            std::vector<std::vector<uint16_t>> planes(L + 1);
            std::vector<std::vector<int>> eA(L + 1);
            size_t bytes = 0;
            std::vector<size_t> offP(L + 1, 0);
            for (int l = 2; l <= L; ++l) {
                const int n = dsc->width[l - 1], np = dsc->width[l - 2];
                const int fan = np + (l == dsc->skip_layer ? in_dim : 0);
                oz_slice_weights(dsc->W[l - 1], n, np, fan, planes[l], eA[l]);
                offP[l] = bytes;
                bytes += planes[l].size() * 2;
                bytes = (bytes + 255) & ~(size_t)255;
                nh.oz_off_eA[l] = bytes;
                bytes += eA[l].size() * 4;
                bytes = (bytes + 255) & ~(size_t)255;
            }
            CU(cudaMalloc(&nh.ozblob, bytes));
            unsigned char *db = reinterpret_cast<unsigned char *>(nh.ozblob);
            nh.ozmap.assign(L + 1, NetHost::MapBytes{});
            for (int l = 2; l <= L; ++l) {
                CU(cudaMemcpy(db + offP[l], planes[l].data(), planes[l].size() * 2, cudaMemcpyHostToDevice));
                CU(cudaMemcpy(db + nh.oz_off_eA[l], eA[l].data(), eA[l].size() * 4, cudaMemcpyHostToDevice));
                CU(oz_encode_weights(nh.ozmap[l].b, db + offP[l], dsc->width[l - 1], dsc->width[l - 2]));
            }
        }
    }
    nh.N = N;
    nh.max_w = mw;
    CU(cudaMemcpyAsync(ctx->d_nets + id, &nd, sizeof(NetDev), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->nets.push_back(nh);
    ctx->max_n_loaded = std::max(ctx->max_n_loaded, N);
    ctx->max_w_loaded = std::max(ctx->max_w_loaded, mw);
    *net_id = id;
    return AM_OK;
}

am_status am_reset(am_ctx *ctx)
{
    if (!ctx || !ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "no context");
    CU(cudaMemsetAsync(ctx->ar.slots, 0, sizeof(unsigned long long) * (ctx->ar.slot_mask + 1), ctx->stream));
    CU(cudaMemsetAsync(ctx->ar.counters, 0, sizeof(unsigned long long) * kNumCounters, ctx->stream));
    CU(cudaMemsetAsync(ctx->ar.ready, 0, sizeof(unsigned) * ctx->ar.cap, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->solved_upto = 0;
    ctx->stats = am_stats_t{};
    ctx->mesh_valid = false;
    ctx->timed_out = false;
    ctx->test_stall_ids = 0;
    ctx->test_wait_ns = 0;
    return AM_OK;
}

am_status am_release_nets(am_ctx *ctx)
{
    am_status s = am_reset(ctx);
    if (s != AM_OK) return s;
    for (auto &n : ctx->nets) {
        if (n.blob) CU(cudaFree(n.blob));
        if (n.fblob) CU(cudaFree(n.fblob));
        if (n.tblob) CU(cudaFree(n.tblob));
        if (n.ozblob) CU(cudaFree(n.ozblob));
    }
    ctx->nets.clear();
    ctx->mesh.clear();
    ctx->max_n_loaded = ctx->max_w_loaded = 1;
    return AM_OK;
}

// Capacity of the seed buffers for n rays (rays: origins then dirs, n x 3 each at a stride of
// seed_cap rows).
static am_status ensure_seed_cap(am_ctx *ctx, int n)
{
    if (n <= ctx->seed_cap) return AM_OK;
    if (ctx->d_rays) cudaFree(ctx->d_rays);
    if (ctx->d_seed_keys) cudaFree(ctx->d_seed_keys);
    if (ctx->d_seed_x) cudaFree(ctx->d_seed_x);
    if (ctx->d_seed_ok) cudaFree(ctx->d_seed_ok);
    ctx->d_rays = nullptr; ctx->d_seed_keys = nullptr; ctx->d_seed_x = nullptr; ctx->d_seed_ok = nullptr;
    ctx->seed_cap = 0;
    CU(cudaMalloc(&ctx->d_rays, sizeof(double) * 6 * n));
    CU(cudaMalloc(&ctx->d_seed_keys, sizeof(unsigned long long) * ctx->ar.kw * n));
    CU(cudaMalloc(&ctx->d_seed_x, sizeof(double) * 3 * n));
    CU(cudaMalloc(&ctx->d_seed_ok, sizeof(int) * (n + 2)));
    ctx->seed_cap = n;
    return AM_OK;
}

// Dichotomy on n_rays device segments o + t d, t in [0, R] (origins at d_rays, dirs at
// d_rays + 3 seed_cap), then the push of the new seed cells.  h_points (may be NULL): the
// seed point of every segment, NaN where it produced none.
static am_status run_seed(am_ctx *ctx, int net_id, int n_rays, double R, int *n_seeded, double *h_points)
{
    unsigned long long *d_new = ctx->d_netcnt + 5 * kMaxNets;
    CU(cudaMemsetAsync(d_new, 0, sizeof(unsigned long long), ctx->stream));
    SeedArgs a{};
    a.nets = ctx->d_nets;
    a.ar = ctx->ar;
    a.net = net_id;
    a.n_rays = n_rays;
    a.origins = ctx->d_rays;
    a.dirs = ctx->d_rays + 3 * (size_t)ctx->seed_cap;
    a.R = R;
    a.max_halvings = 200;
    a.max_n = ctx->opts.max_neurons;
    a.max_w = ctx->opts.max_width;
    a.seed_keys = ctx->d_seed_keys;
    a.seed_x = ctx->d_seed_x;
    a.seed_ok = ctx->d_seed_ok;
    a.n_new = d_new;
    a.df = ctx->nets[net_id].dev.fp64_only ? 0 : 1;
    launch_seed(a, ctx->stream);
    CU(cudaGetLastError());
    ctx->stats.kernel_launches += 2;
    unsigned long long hn = 0;
    CU(cudaMemcpyAsync(&hn, d_new, sizeof hn, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<int> ok(n_rays);
    CU(cudaMemcpyAsync(ok.data(), ctx->d_seed_ok, sizeof(int) * n_rays, cudaMemcpyDeviceToHost, ctx->stream));
    if (h_points)
        CU(cudaMemcpyAsync(h_points, ctx->d_seed_x, sizeof(double) * 3 * n_rays, cudaMemcpyDeviceToHost,
                           ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (h_points)
        for (int r = 0; r < n_rays; ++r)
            if (ok[r] != 1) h_points[3 * r] = h_points[3 * r + 1] = h_points[3 * r + 2] = std::nan("");
    if (n_seeded) *n_seeded = (int)hn;
    ctx->mesh_valid = false;
    if (hn == 0) {
        int nosign = 0;
        for (int v : ok) nosign += v == -4;
        return fail(ctx, AM_ERR_NO_SEED_CELL, "no new seed cell (%d of %d segments without a sign change)", nosign,
                    n_rays);
    }
    return AM_OK;
}

am_status am_seed(am_ctx *ctx, int net_id, const double *h_origins, const double *h_dirs, int n_rays, double R,
                  int *n_seeded)
{
    if (!ctx || !ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "no context");
    if (ctx->timed_out) return fail(ctx, AM_ERR_STATE, "a device wait timed out: call am_reset first");
    if (net_id < 0 || net_id >= (int)ctx->nets.size()) return fail(ctx, AM_ERR_INVALID_ARG, "unknown net %d", net_id);
    if (!h_origins || !h_dirs || n_rays < 1 || !(R > 0.0)) return fail(ctx, AM_ERR_INVALID_ARG, "bad rays");
    am_status s = ensure_seed_cap(ctx, n_rays);
    if (s != AM_OK) return s;
    CU(cudaMemcpyAsync(ctx->d_rays, h_origins, sizeof(double) * 3 * n_rays, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->d_rays + 3 * (size_t)ctx->seed_cap, h_dirs, sizeof(double) * 3 * n_rays,
                       cudaMemcpyHostToDevice, ctx->stream));
    return run_seed(ctx, net_id, n_rays, R, n_seeded, nullptr);
}

am_status am_seed_sphere_trace(am_ctx *ctx, int net_id, const double *h_starts, int n_starts, double eta,
                               int max_steps, double eps, int *n_seeded, double *h_seed_points)
{
    if (!ctx || !ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "no context");
    if (net_id < 0 || net_id >= (int)ctx->nets.size()) return fail(ctx, AM_ERR_INVALID_ARG, "unknown net %d", net_id);
    if (!h_starts || n_starts < 1 || n_starts > kMaxTriggerPoints) return fail(ctx, AM_ERR_INVALID_ARG, "bad starts");
    if (!(eta > 0.0 && eta <= 1.0) || max_steps < 0 || max_steps > kMaxTraceSteps || !(eps >= 0.0) ||
        !std::isfinite(eps))
        return fail(ctx, AM_ERR_INVALID_ARG, "bad tracing parameters (0 < eta <= 1, 0 <= max_steps <= %d, eps >= 0)",
                    kMaxTraceSteps);
    am_status s = ensure_seed_cap(ctx, n_starts);
    if (s != AM_OK) return s;
    CU(grow(&ctx->d_trig, &ctx->trig_cap, 3 * (int64_t)n_starts));
    CU(cudaMemcpyAsync(ctx->d_trig, h_starts, sizeof(double) * 3 * n_starts, cudaMemcpyHostToDevice, ctx->stream));
    TraceArgs t{};
    t.nets = ctx->d_nets;
    t.net = net_id;
    t.n = n_starts;
    t.starts = ctx->d_trig;
    t.eta = eta;
    t.eps = eps;
    t.pad = kTracePad;
    t.max_steps = max_steps;
    t.max_n = ctx->opts.max_neurons;
    t.max_w = ctx->opts.max_width;
    t.origins = ctx->d_rays;
    t.dirs = ctx->d_rays + 3 * (size_t)ctx->seed_cap;
    launch_trace(t, ctx->stream);
    CU(cudaGetLastError());
    ctx->stats.kernel_launches += 1;
    return run_seed(ctx, net_id, n_starts, 1.0, n_seeded, h_seed_points);
}

am_status am_seed_pairs(am_ctx *ctx, int net_id, const double *h_points, int n_points, int max_pairs, int *n_pairs,
                        int *n_seeded, double *h_seed_points)
{
    if (!ctx || !ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "no context");
    if (net_id < 0 || net_id >= (int)ctx->nets.size()) return fail(ctx, AM_ERR_INVALID_ARG, "unknown net %d", net_id);
    if (!h_points || n_points < 1 || n_points > kMaxTriggerPoints || max_pairs < 1 || max_pairs > kMaxTriggerPoints)
        return fail(ctx, AM_ERR_INVALID_ARG, "bad samples (1 <= n_points, max_pairs <= %d)", kMaxTriggerPoints);
    am_status s = ensure_seed_cap(ctx, max_pairs);
    if (s != AM_OK) return s;
    // samples (3 n), F (n), then the two index lists (2 max_pairs ints in max_pairs doubles)
    CU(grow(&ctx->d_trig, &ctx->trig_cap, 4 * (int64_t)n_points + max_pairs + 1));
    CU(cudaMemcpyAsync(ctx->d_trig, h_points, sizeof(double) * 3 * n_points, cudaMemcpyHostToDevice, ctx->stream));
    int *d_np = ctx->d_seed_ok + ctx->seed_cap;
    PairArgs p{};
    p.nets = ctx->d_nets;
    p.net = net_id;
    p.n_points = n_points;
    p.max_pairs = max_pairs;
    p.points = ctx->d_trig;
    p.F = ctx->d_trig + 3 * (size_t)n_points;
    p.neg_idx = (int *)(ctx->d_trig + 4 * (size_t)n_points);
    p.pos_idx = p.neg_idx + max_pairs;
    p.max_n = ctx->opts.max_neurons;
    p.max_w = ctx->opts.max_width;
    p.origins = ctx->d_rays;
    p.dirs = ctx->d_rays + 3 * (size_t)ctx->seed_cap;
    p.n_pairs = d_np;
    p.df = ctx->nets[net_id].dev.fp64_only ? 0 : 1;
    launch_pairs(p, ctx->stream);
    CU(cudaGetLastError());
    ctx->stats.kernel_launches += 2;
    int hp = 0;
    CU(cudaMemcpyAsync(&hp, d_np, sizeof hp, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (n_pairs) *n_pairs = hp;
    if (h_seed_points)
        for (int i = 0; i < 3 * max_pairs; ++i) h_seed_points[i] = std::nan("");
    if (hp == 0) {
        if (n_seeded) *n_seeded = 0;
        return fail(ctx, AM_ERR_NO_SEED_CELL, "no pair of samples with F of opposite signs");
    }
    return run_seed(ctx, net_id, hp, 1.0, n_seeded, h_seed_points);
}

static am_status assemble(am_ctx *ctx, int64_t n_cells)
{
    const int nn = (int)ctx->nets.size();
    unsigned long long *cnt = ctx->d_netcnt;
    AsmArgs a{};
    a.ar = ctx->ar;
    a.nets = ctx->d_nets;
    a.n_cells = n_cells;
    a.n_nets = nn;
    a.face_count = cnt;
    a.face_fill = cnt + kMaxNets;
    a.face_base = cnt + 2 * kMaxNets;
    a.vert_count = cnt + 3 * kMaxNets;
    a.vert_base = cnt + 4 * kMaxNets;
    CU(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 2 * kMaxNets, ctx->stream));
    CU(cudaMemsetAsync(a.vert_count, 0, sizeof(unsigned long long) * kMaxNets, ctx->stream));
    launch_asm_count(a, ctx->stream);
    std::vector<unsigned long long> fc(nn), base(nn);
    CU(cudaMemcpyAsync(fc.data(), a.face_count, sizeof(unsigned long long) * nn, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    int64_t nf = 0;
    for (int i = 0; i < nn; ++i) { base[i] = nf; nf += (int64_t)fc[i]; }
    CU(cudaMemcpyAsync(a.face_base, base.data(), sizeof(unsigned long long) * nn, cudaMemcpyHostToDevice, ctx->stream));
    CU(grow(&ctx->d_perm, &ctx->faces_cap, nf + 1));
    CU(grow(&ctx->d_coff, &ctx->coff_cap, nf + 2));
    const int64_t blocks = (nf + 4095) / 4096 + 1;
    CU(grow(&ctx->d_scan_tmp, &ctx->scan_tmp_len, 2 * blocks + 4));
    a.perm = ctx->d_perm;
    a.corner_off = ctx->d_coff;
    a.n_faces = nf;
    launch_asm_scatter(a, ctx->stream);
    CU(cudaGetLastError());
    CU(launch_asm_offsets(a, ctx->d_scan_tmp, ctx->scan_tmp_len, ctx->stream));
    int64_t ncorner = 0;
    CU(cudaMemcpyAsync(&ncorner, ctx->d_coff + nf, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (ncorner + 1 > ctx->corners_cap) {     // the three per-corner arrays grow together
        int64_t c1 = 0, c2 = 0, c3 = 0;
        CU(grow(&ctx->d_cvid, &c1, ncorner + 1));
        CU(grow(&ctx->d_fv, &c2, ncorner + 1));
        CU(grow(&ctx->d_fe, &c3, ncorner + 1));
        ctx->corners_cap = std::min(c1, std::min(c2, c3));
    }
    CU(grow(&ctx->d_xyz, &ctx->verts_cap, 3 * (ncorner + 1)));
    CU(grow(&ctx->d_fkeys, &ctx->fkeys_cap, (nf + 1) * ctx->ar.kw));
    const int64_t vs = pow2_at_least(std::max<int64_t>(2 * ncorner, 1024));
    if (vs > ctx->vslots_n) {
        if (ctx->d_vslots) cudaFree(ctx->d_vslots);
        ctx->d_vslots = nullptr;
        CU(cudaMalloc(&ctx->d_vslots, sizeof(unsigned long long) * vs));
        ctx->vslots_n = vs;
    }
    CU(cudaMemsetAsync(ctx->d_vslots, 0, sizeof(unsigned long long) * ctx->vslots_n, ctx->stream));
    a.corner_vid = ctx->d_cvid;
    a.vslots = ctx->d_vslots;
    a.vslot_mask = (unsigned long long)(ctx->vslots_n - 1);
    a.out_xyz = ctx->d_xyz;
    a.out_fv = ctx->d_fv;
    a.out_edges = ctx->d_fe;
    a.out_keys = ctx->d_fkeys;
    launch_asm_vertices(a, ctx->stream);
    launch_asm_lookup(a, ctx->stream);
    CU(cudaGetLastError());
    std::vector<unsigned long long> vc(nn), vb(nn);
    CU(cudaMemcpyAsync(vc.data(), a.vert_count, sizeof(unsigned long long) * nn, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    int64_t nvtx = 0;
    for (int i = 0; i < nn; ++i) { vb[i] = nvtx; nvtx += (int64_t)vc[i]; }
    CU(cudaMemcpyAsync(a.vert_base, vb.data(), sizeof(unsigned long long) * nn, cudaMemcpyHostToDevice, ctx->stream));
    launch_asm_write(a, ctx->stream);
    CU(cudaGetLastError());
    // per-net corner ranges
    std::vector<int64_t> coff_at(nn + 1);
    ctx->mesh.assign(nn, MeshInfo{});
    for (int i = 0; i <= nn; ++i) {
        const int64_t f = i < nn ? (int64_t)base[i] : nf;
        CU(cudaMemcpyAsync(&coff_at[i], ctx->d_coff + f, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < nn; ++i) {
        MeshInfo &m = ctx->mesh[i];
        m.faces = (int64_t)fc[i];
        m.face_base = (int64_t)base[i];
        m.corner_base = coff_at[i];
        m.corners = coff_at[i + 1] - coff_at[i];
        m.verts = (int64_t)vc[i];
        m.vert_base = (int64_t)vb[i];
    }
    ctx->stats.kernel_launches += nf > 0 ? 8 : 6;
    ctx->stats.faces = nf;
    ctx->stats.corners = ncorner;
    ctx->stats.vertices = nvtx;
    ctx->mesh_valid = true;
    return AM_OK;
}

// Per-item scratch of the rank-1 compose (a batch of up to 4 x batch_cells children) and the
// classification counters.
static am_status ensure_r1_scratch(am_ctx *ctx)
{
    R1Scratch &r = ctx->r1;
    if (r.counts) return AM_OK;
    const int64_t items = 4 * ctx->oz.batch_cells;
    CU(cudaMalloc(&r.counts, sizeof(unsigned long long) * (kMaxLayers + 1)));
    CU(cudaMalloc(&r.offs, sizeof(int) * 2 * (kMaxLayers + 1)));
    CU(cudaMalloc(&r.it_l, sizeof(int) * items));
    CU(cudaMalloc(&r.it_k, sizeof(int) * items));
    CU(cudaMalloc(&r.it_a, sizeof(float) * 8 * items));
    r.item_cap = items;
    CU(cudaMalloc(&ctx->fb_list, sizeof(int32_t) * ctx->oz.batch_cells));
    CU(cudaMalloc(&ctx->fb_count, sizeof(unsigned long long)));
    CU(cudaMalloc(&ctx->clip_work, sizeof(unsigned long long)));
    CU(cudaMalloc(&ctx->chk, sizeof(CheckRec) * ctx->oz.batch_cells));
    CU(cudaMalloc(&ctx->chk_count, sizeof(unsigned long long)));
    CU(cudaMalloc(&ctx->chk_status, sizeof(int) * ctx->oz.batch_cells));
    return AM_OK;
}

// Level rows (FP32 pairs) for at least n cells in buffer b, keeping the other buffer (the parents).
static am_status ensure_level_rows(am_ctx *ctx, int b, int64_t n)
{
    if (ctx->lv_cap[b] >= n && ctx->lv_rows[b]) return AM_OK;
    if (ctx->lv_rows[b]) CU(cudaFree(ctx->lv_rows[b]));
    ctx->lv_rows[b] = nullptr;
    ctx->lv_cap[b] = 0;
    const int64_t cap = std::max<int64_t>(n + n / 4, 4096);
    CU(cudaMalloc(&ctx->lv_rows[b], sizeof(double) * 4 * (int64_t)(ctx->nets[0].N + 1) * cap));
    ctx->lv_cap[b] = cap;
    return AM_OK;
}

// One breadth-first level [f0, f1) of the AM_PREC_SLICED march.  The level's rows are composed on
// the tensor cores into the level buffer: in full for the cells classified so (and for every
// cell of the first level of a call), by the rank-1 update from the previous level's rows for the
// others.  Then the learned proposal's scores (tensor cores) and the clip (certified FP32 tests on
// the rows, FP64 where they do not decide), per chunk of the level: the whole level in one chunk
// with the warp clip, batches of oz.batch_cells with the tensor-core check or the block clip; and
// finally the classification of the cells this level pushed.  Events: oz_ev[0..1] the compose,
// then three per chunk; *nchunks receives the chunk count.
static am_status sliced_level(am_ctx *ctx, MarchArgs &ma, int64_t f0, int64_t f1, bool prop_tc, int *nchunks)
{
    const NetHost &nh = ctx->nets[0];
    const OzNet view = oz_view(nh);
    const int L = nh.dev.L, N = nh.dev.N;
    const int64_t nl = f1 - f0;
    const int64_t chunk = ctx->oz.batch_cells;           // the compose's batch
    const bool warp_clip = ctx->clip_kernel == 0 && ma.candidates != kCandNone && N <= kMaxNeurons;
    // the proposal and the clip take the whole level in one launch each (the warp clip draws its
    // cells from a counter), except with the tensor-core check, whose records hold one batch
    const int64_t cchunk = warp_clip && ctx->check_kernel != 1 ? std::max<int64_t>(nl, 1) : chunk;
    const int nchunk = (int)((nl + cchunk - 1) / cchunk);
    while ((int)ctx->oz_ev.size() < 2 + 3 * nchunk) {
        cudaEvent_t e = nullptr;
        CU(cudaEventCreate(&e));
        ctx->oz_ev.push_back(e);
    }
    const int cur = ctx->stats.levels & 1;              // this level's buffer; the other holds its parents
    am_status s = ensure_level_rows(ctx, cur, nl);
    if (s != AM_OK) return s;
    R1Scratch &r = ctx->r1;
    if (r.list_cap < nl) {
        if (r.full_list) CU(cudaFree(r.full_list));
        if (r.r1_list) CU(cudaFree(r.r1_list));
        r.full_list = r.r1_list = nullptr;
        r.list_cap = 0;
        const int64_t cap = std::max<int64_t>(nl + nl / 4, 4096);
        CU(cudaMalloc(&r.full_list, sizeof(int32_t) * cap));
        CU(cudaMalloc(&r.r1_list, sizeof(int32_t) * cap));
        // the warp clip's fallback cells of the whole level
        if (ctx->fb_list) CU(cudaFree(ctx->fb_list));
        ctx->fb_list = nullptr;
        CU(cudaMalloc(&ctx->fb_list, sizeof(int32_t) * cap));
        r.list_cap = cap;
    }
    if (warp_clip) CU(cudaMemsetAsync(ctx->fb_count, 0, sizeof(unsigned long long), ctx->stream));
    if (prop_tc) CU(prop_tc_grow(ctx->prop.tc, (int)cchunk));
    const int period = ctx->oz_rank1_period > 0 ? ctx->oz_rank1_period : 32;
    int64_t launches = 0;
    cudaEvent_t *ev = ctx->oz_ev.data();
    CU(cudaEventRecord(ev[0], ctx->stream));
    double *rows = ctx->lv_rows[cur];
    const unsigned long long *c = ctx->r1_hcounts;
    int h_offs[2 * (kMaxLayers + 1)] = {};
    int64_t acc = 0, cnt_le[kMaxLayers + 1] = {};
    for (int l = 1; l <= L; ++l) {
        h_offs[l] = (int)acc;
        acc += (int64_t)c[l];
        cnt_le[l] = acc;
    }
    const int64_t n_full = (int64_t)c[0], n_r1 = acc;
    // the plan covers the whole next level; a level cut short by max_cells is composed in full
    if (ctx->r1_planned && n_full + n_r1 == nl) {
        // the previous level classified these cells: full list and rank-1 list (by flip layer)
        CU(oz_rank1_scatter(ctx->ar, f0, f1, h_offs, L, r, ctx->stream));
        launches += 1;
        if (n_full > 0) {
            CU(oz_compose(view, ctx->ar.keys, ctx->ar.kw, n_full, rows, true, ctx->oz, ctx->oz_tile_cells,
                          ctx->sm_count, ctx->stream, r.full_list, f0));
            launches += (2 * (int64_t)L - 1) * ((n_full + chunk - 1) / chunk);
        }
        if (n_r1 > 0) {
            const R1Cells cells{ctx->ar.keys, ctx->ar.kw, ctx->ar.parent, ctx->ar.entry_plane};
            CU(oz_rank1(view, cells, r.r1_list, n_r1, cnt_le, ctx->lv_rows[cur ^ 1], ctx->r1_prev0, rows, f0, ctx->oz, r,
                        ctx->oz_tile_cells, ctx->sm_count, ctx->stream));
            launches += 2 * (int64_t)L * ((n_r1 + 4 * chunk - 1) / (4 * chunk));
        }
    } else {
        // every cell in full; their chains of rank-1 composes start here
        CU(cudaMemsetAsync(ctx->ar.chain + f0, 0, sizeof(int32_t) * nl, ctx->stream));
        CU(oz_compose(view, ctx->ar.keys + f0 * ctx->ar.kw, ctx->ar.kw, nl, rows, true, ctx->oz, ctx->oz_tile_cells,
                      ctx->sm_count, ctx->stream));
        launches += (2 * (int64_t)L - 1) * ((nl + chunk - 1) / chunk);
    }
    CU(cudaEventRecord(ev[1], ctx->stream));
    const int64_t rstride = 8 * (int64_t)(N + 1);         // floats per cell
    for (int b = 0; b < nchunk; ++b) {
        const int64_t c0 = f0 + b * cchunk, c1 = std::min<int64_t>(f1, c0 + cchunk);
        CU(cudaEventRecord(ev[2 + 3 * b], ctx->stream));
        ma.scores_in = nullptr;
        if (prop_tc) {
            const NetDev &nd = nh.dev;
            PropFeatures pf{};
            pf.keys = ctx->ar.keys;
            pf.kw = ctx->ar.kw;
            pf.entry_pt = ctx->ar.entry_pt;
            pf.c0 = c0;
            pf.n = c1 - c0;
            pf.rows = reinterpret_cast<const float *>(rows) + (c0 - f0) * rstride;
            pf.rstride = rstride;
            pf.N = nd.N;
            pf.L = nd.L;
            for (int l = 0; l <= nd.L; ++l) { pf.row0[l] = nd.row0[l]; pf.width[l] = nd.width[l]; }
            ProposalDev &pd = ctx->prop;
            CU(prop_tc_features(pd.tc, pf, ctx->stream));
            CU(prop_tc_forward(pd.tc, pd.w + pd.off[1], pd.w + pd.off[3], pd.w + pd.off[5], (int)(c1 - c0), pd.tc.scores,
                               false, pd.n_out, ctx->oz.err, ctx->stream));
            launches += 4;
            ma.scores_in = pd.tc.scores;
            ma.scores_ld = pd.n_out;
        }
        CU(cudaEventRecord(ev[3 + 3 * b], ctx->stream));
        ma.begin = c0;
        ma.end = c1;
        ma.rows_in = reinterpret_cast<const float *>(rows) + (c0 - f0) * rstride;
        if (warp_clip) {
            // one warp per cell; the cells it cannot decide outright go to the block kernel, once
            // for the whole level after its last chunk
            ma.fb_list = ctx->fb_list;
            ma.fb_count = ctx->fb_count;
            if (ctx->check_kernel == 1) {
                // candidate clip in the warp, the dense check on the tensor cores, then emit and push
                CU(cudaMemsetAsync(ctx->chk_count, 0, sizeof(unsigned long long), ctx->stream));
                ma.chk = ctx->chk;
                ma.chk_count = ctx->chk_count;
                ma.chk_status = ctx->chk_status;
                launch_clip_warp(ma, ctx->stream);
                CU(cudaGetLastError());
                CheckArgs ca{};
                ca.rec = ctx->chk;
                ca.count = ctx->chk_count;
                ca.rows = reinterpret_cast<const float *>(ma.rows_in);
                ca.begin = c0;
                ca.N = N;
                ca.box = ma.box_hi;
                ca.box_lo = ma.box_lo;
                ca.delta = ma.delta;
                ca.status = ctx->chk_status;
                ca.counters = ctx->ar.counters;
                ca.err = ctx->oz.err;
                launch_check_tc(ca, ctx->sm_count, ctx->stream);
                CU(cudaGetLastError());
                launch_clip_warp_finish(ma, ctx->stream);
                CU(cudaGetLastError());
                ma.chk = nullptr;
                ma.chk_count = nullptr;
                ma.chk_status = nullptr;
                ctx->stats.cell_launches += 2;
                launches += 2;
            } else {
                CU(cudaMemsetAsync(ctx->clip_work, 0, sizeof(unsigned long long), ctx->stream));
                ma.work = ctx->clip_work;
                launch_clip_warp(ma, ctx->stream);
                CU(cudaGetLastError());
                ma.work = nullptr;
            }
            ctx->stats.cell_launches += 1;
            launches += 1;
            if (b == nchunk - 1) {
                // the level's fallback cells: rows from the level's buffer, nearest candidates (with
                // several chunks the proposal's scores cover the last one only; the candidates never
                // change the face)
                MarchArgs mb = ma;
                mb.begin = f0;
                mb.end = f1;
                mb.rows_in = rows;
                mb.scores_in = nullptr;
                if (mb.candidates == kCandLearned) mb.candidates = kCandNearest;
                mb.list = ctx->fb_list;
                mb.list_count = ctx->fb_count;
                launch_march(mb, 1, false, (int)std::min<int64_t>(nl, 2 * (int64_t)ctx->sm_count), ctx->stream);
                CU(cudaGetLastError());
                ctx->stats.cell_launches += 1;
                launches += 1;
            }
        } else {
            launch_march(ma, 1, false, (int)(c1 - c0), ctx->stream);   // certified FP32 tests on the pairs
            CU(cudaGetLastError());
            ctx->stats.cell_launches += 1;
            launches += 1;
        }
        CU(cudaEventRecord(ev[4 + 3 * b], ctx->stream));
    }
    // classify the cells this level pushed (the next level) for the rank-1 compose
    ctx->r1_planned = false;
    if (period > 1) {
        CU(oz_rank1_classify(view, ctx->ar, f0, f1, f1, period, r, ctx->stream));
        CU(cudaMemcpyAsync(ctx->r1_hcounts, r.counts, sizeof(unsigned long long) * (kMaxLayers + 1),
                           cudaMemcpyDeviceToHost, ctx->stream));
        launches += 1;
        ctx->r1_planned = true;
        ctx->r1_prev0 = f0;
    }
    ctx->stats.kernel_launches += launches;
    *nchunks = nchunk;
    return AM_OK;
}

am_status am_march(am_ctx *ctx, const am_march_opts *o)
{
    if (!ctx || !ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "no context");
    if (ctx->nets.empty()) return fail(ctx, AM_ERR_STATE, "no net loaded");
    if (ctx->timed_out) return fail(ctx, AM_ERR_STATE, "a device wait timed out: call am_reset first");
    am_march_opts op{};
    if (o) op = *o;
    if (!(op.box > 0.0)) op.box = 1.5;
    if (!(op.delta > 0.0)) op.delta = 1e-10;
    if (op.precision == AM_PREC_TENSOR)
        return fail(ctx, AM_ERR_INVALID_ARG, "AM_PREC_TENSOR rows carry error estimates, not bounds: the "
                    "march takes AM_PREC_FP64, AM_PREC_MIXED or AM_PREC_SLICED (am_compose takes all four)");
    if (op.precision != AM_PREC_FP64 && op.precision != AM_PREC_MIXED && op.precision != AM_PREC_SLICED)
        return fail(ctx, AM_ERR_INVALID_ARG, "unknown precision %d", (int)op.precision);
    const bool sliced = op.precision == AM_PREC_SLICED;
    if (sliced) {
        // the tensor-core compose runs per net over a batch of cells: one net per march
        if (ctx->nets.size() != 1)
            return fail(ctx, AM_ERR_INVALID_ARG, "AM_PREC_SLICED marches one net (context holds %d)",
                        (int)ctx->nets.size());
        if (!ctx->nets[0].oz_ok)
            return fail(ctx, AM_ERR_INVALID_ARG, "AM_PREC_SLICED needs a ReLU net with every hidden fan-in <= %d",
                        kOzMaxFanIn);
        op.schedule = AM_SCHED_LEVELS;
        am_status se = ensure_oz_scratch(ctx);
        if (se != AM_OK) return se;
        se = ensure_r1_scratch(ctx);
        if (se != AM_OK) return se;
        ctx->r1_planned = false;     // the first level of a call is composed in full
    }
    if (op.schedule != AM_SCHED_PERSISTENT && op.schedule != AM_SCHED_LEVELS)
        return fail(ctx, AM_ERR_INVALID_ARG, "unknown schedule %d", (int)op.schedule);
    if (op.max_cells < 0 || op.grid_blocks < 0) return fail(ctx, AM_ERR_INVALID_ARG, "negative limit");
    const int64_t stall = ctx->test_stall_ids;
    const long long wait_ns = ctx->test_wait_ns > 0 ? ctx->test_wait_ns : kWaitNs;
    ctx->test_stall_ids = 0;             // the hook applies to this one march
    ctx->test_wait_ns = 0;
    if (stall > 0 && (op.schedule != AM_SCHED_PERSISTENT || sliced))
        return fail(ctx, AM_ERR_INVALID_ARG, "am_test_stall_next_march needs the persistent schedule");
    const int mode = op.precision == AM_PREC_MIXED ? 1 : 0;   // kDF only for the double-float path
    unsigned long long hc[kNumCounters];
    am_status s = sync_status(ctx, hc);
    if (s != AM_OK) return s;
    MarchArgs ma{};
    ma.nets = ctx->d_nets;
    ma.ar = ctx->ar;
    ma.box = op.box;
    ma.box_hi = (float)op.box;
    ma.box_lo = (float)(op.box - (double)ma.box_hi);
    ma.delta = op.delta;
    ma.max_n = ctx->opts.max_neurons;
    ma.max_w = ctx->opts.max_width;
    ma.wait_ns = wait_ns;
    if (op.candidates != AM_CAND_NEAREST && op.candidates != AM_CAND_LEARNED && op.candidates != AM_CAND_NONE)
        return fail(ctx, AM_ERR_INVALID_ARG, "unknown candidates mode %d", (int)op.candidates);
    if (op.candidates == AM_CAND_LEARNED && !ctx->prop.w)
        return fail(ctx, AM_ERR_STATE, "AM_CAND_LEARNED needs a proposal (am_proposal_init / am_proposal_train)");
    if (op.candidates == AM_CAND_LEARNED && ctx->prop.hidden > proposal_max_hidden())
        return fail(ctx, AM_ERR_INVALID_ARG, "proposal hidden width %d above the march's %d", ctx->prop.hidden,
                    proposal_max_hidden());
    ma.candidates = (int)op.candidates;
    if (ctx->prop.w) {
        ProposalDev &p = ctx->prop;
        ma.prop.w1 = p.wb + p.off[0];
        ma.prop.b1 = p.w + p.off[1];
        ma.prop.w2t = p.w2t;
        ma.prop.b2 = p.w + p.off[3];
        ma.prop.w3t = p.w3t;
        ma.prop.b3 = p.w + p.off[5];
        ma.prop.n_in = p.n_in;
        ma.prop.hidden = p.hidden;
        ma.prop.n_out = p.n_out;
    }
    // learned candidates on the sliced level march: the proposal's forward pass per batch on
    // the tensor cores (the march kernel then reads the scores)
    const bool prop_tc = sliced && op.candidates == AM_CAND_LEARNED && ctx->prop.tc.ok &&
                         ctx->prop.n_out == ctx->nets[0].N && ctx->prop.n_in == 7 + ctx->nets[0].dev.L &&
                         ctx->oz.batch_cells <= ctx->prop.tc.max_rows;
    const int64_t start = ctx->solved_upto;
    const int64_t limit = op.max_cells > 0 ? std::min<int64_t>(start + op.max_cells, ctx->ar.cap) : ctx->ar.cap;
    bool incomplete = false;
    CU(cudaEventRecord(ctx->ev0, ctx->stream));
    if (op.schedule == AM_SCHED_PERSISTENT) {
        // tickets restart at the first unsolved cell; every earlier cell counts as done
        const unsigned long long hs = (unsigned long long)start;
        CU(cudaMemcpyAsync(ctx->ar.counters + kHead, &hs, sizeof hs, cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemcpyAsync(ctx->ar.counters + kDone, &hs, sizeof hs, cudaMemcpyHostToDevice, ctx->stream));
        if (stall > 0) {
            // ids handed out and never published (their ready flags stay 0 until am_reset): the
            // blocks that take these tickets wait until the limit and report the time-out
            const unsigned long long n = (unsigned long long)std::min<int64_t>((int64_t)hc[kNCells] + stall, ctx->ar.cap);
            CU(cudaMemcpyAsync(ctx->ar.counters + kNCells, &n, sizeof n, cudaMemcpyHostToDevice, ctx->stream));
        }
        ma.limit = limit;
        int grid = ctx->sm_count * ctx->blocks_per_sm;
        if (op.grid_blocks > 0) grid = std::min(grid, op.grid_blocks);
        CU(cudaEventRecord(ctx->evk0, ctx->stream));
        launch_march(ma, mode, true, grid, ctx->stream);
        CU(cudaGetLastError());
        CU(cudaEventRecord(ctx->evk1, ctx->stream));
        ctx->stats.cell_launches += 1;
        ctx->stats.kernel_launches += 1;
        s = sync_status(ctx, hc);
        if (s != AM_OK) return s;
        float kms = 0.f;
        CU(cudaEventElapsedTime(&kms, ctx->evk0, ctx->evk1));
        ctx->stats.ms_cell_kernels += kms;
        const int64_t n = std::min<int64_t>((int64_t)hc[kNCells], ctx->ar.cap);
        ctx->solved_upto = std::min<int64_t>(n, limit);
        incomplete = op.max_cells > 0 && (int64_t)hc[kNCells] > ctx->solved_upto;
    } else {
        int64_t f0 = start, f1 = std::min<int64_t>((int64_t)hc[kNCells], ctx->ar.cap);
        while (f0 < f1) {
            if (f0 >= limit) { incomplete = true; break; }
            f1 = std::min<int64_t>(f1, limit);
            CU(cudaEventRecord(ctx->evk0, ctx->stream));
            int nbatch = 0;
            if (sliced) {
                s = sliced_level(ctx, ma, f0, f1, prop_tc, &nbatch);
                if (s != AM_OK) return s;
            } else {
                ma.begin = f0;
                ma.end = f1;
                launch_march(ma, mode, false, (int)std::min<int64_t>(f1 - f0, 1 << 20), ctx->stream);
                CU(cudaGetLastError());
                ctx->stats.cell_launches += 1;
                ctx->stats.kernel_launches += 1;
            }
            CU(cudaEventRecord(ctx->evk1, ctx->stream));
            ctx->stats.levels += 1;
            s = sync_status(ctx, hc);
            if (s != AM_OK) return s;
            if (sliced) {
                // events: 0..1 the level's compose, then per chunk of the level: proposal, clip
                float ta = 0.f;
                CU(cudaEventElapsedTime(&ta, ctx->oz_ev[0], ctx->oz_ev[1]));
                ctx->stats.ms_compose += ta;
                for (int b = 0; b < nbatch; ++b) {
                    float tp = 0.f, tb = 0.f;
                    CU(cudaEventElapsedTime(&tp, ctx->oz_ev[2 + 3 * b], ctx->oz_ev[3 + 3 * b]));
                    CU(cudaEventElapsedTime(&tb, ctx->oz_ev[3 + 3 * b], ctx->oz_ev[4 + 3 * b]));
                    ctx->stats.ms_proposal += tp;
                    ctx->stats.ms_clip += tb;
                }
                if (ctx->oz_err_host) {
                    CU(cudaMemsetAsync(ctx->oz.err, 0, sizeof(int), ctx->stream));
                    const size_t pq = sizeof(long long) * 4 * ctx->oz.batch_cells * oz_mp(ctx->opts.max_width);
                    CU(cudaMemsetAsync(ctx->oz.P, 0, pq, ctx->stream));
                    CU(cudaMemsetAsync(ctx->oz.Q, 0, pq, ctx->stream));
                    ctx->oz_dirty = 0;
                    CU(cudaStreamSynchronize(ctx->stream));
                    ctx->timed_out = true;           // the level's rows are not trustworthy
                    ctx->mesh_valid = false;
                    return fail(ctx, AM_ERR_TIMEOUT, "a tensor-core pipeline wait of the sliced compose gave up");
                }
            }
            float kms = 0.f;
            CU(cudaEventElapsedTime(&kms, ctx->evk0, ctx->evk1));
            ctx->stats.ms_cell_kernels += kms;
            if (hc[kStatus] & (kStCellCap | kStHashFull | kStFaceVerts | kStTimeout)) break;
            f0 = f1;
            f1 = std::min<int64_t>((int64_t)hc[kNCells], ctx->ar.cap);
        }
        ctx->solved_upto = f0;
        // keep the ticket counters consistent with the cells solved so far
        const unsigned long long hs = (unsigned long long)f0;
        CU(cudaMemcpyAsync(ctx->ar.counters + kHead, &hs, sizeof hs, cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemcpyAsync(ctx->ar.counters + kDone, &hs, sizeof hs, cudaMemcpyHostToDevice, ctx->stream));
    }
    if (hc[kStatus] & kStTimeout) {
        // a wait gave up: cells may be half written, so no mesh is assembled from them
        ctx->timed_out = true;
        ctx->mesh_valid = false;
        return fail(ctx, AM_ERR_TIMEOUT, "a bounded device wait gave up (after %.3f ms); call am_reset",
                    (double)wait_ns * 1e-6);
    }
    CU(cudaEventRecord(ctx->ev1, ctx->stream));
    s = assemble(ctx, ctx->solved_upto);
    if (s != AM_OK) return s;
    CU(cudaEventRecord(ctx->ev2, ctx->stream));
    s = sync_status(ctx, hc);
    if (s != AM_OK) return s;
    float ms1 = 0.f, ms2 = 0.f;
    cudaEventElapsedTime(&ms1, ctx->ev0, ctx->ev1);
    cudaEventElapsedTime(&ms2, ctx->ev1, ctx->ev2);
    ctx->stats.ms_march += ms1;
    ctx->stats.ms_assemble = ms2;
    ctx->stats.cells = (int64_t)hc[kSolved];
    ctx->stats.empty_faces = (int64_t)hc[kEmpty];
    ctx->stats.degenerate = (int64_t)hc[kDegenerate];
    ctx->stats.refined_cells = (int64_t)hc[kRefined];
    ctx->stats.close_calls = (int64_t)hc[kCloseCalls];
    ctx->stats.fixups = (int64_t)hc[kFixups];
    ctx->stats.cuts = (int64_t)hc[kCuts];
    ctx->stats.clip_fallbacks = (int64_t)hc[kWarpFallback];
    for (int i = 0; i < 10; ++i) ctx->stats.phase_cycles[i] = (int64_t)hc[kPhase0 + i * kCtrStride];
    s = status_error(ctx, hc[kStatus]);
    if (s != AM_OK) return s;
    if (hc[kStatus] & kStClip) ctx->err = "a clip step met an inconsistent polygon (reported as an empty face)";
    return incomplete ? AM_INCOMPLETE : AM_OK;
}

am_status am_compose(am_ctx *ctx, int net_id, const uint64_t *d_keys, int64_t n, am_precision precision,
                     double *d_rows, float *d_err)
{
    if (!ctx || !ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "no context");
    if (net_id < 0 || net_id >= (int)ctx->nets.size()) return fail(ctx, AM_ERR_INVALID_ARG, "unknown net %d", net_id);
    if (n < 0 || (n > 0 && (!d_keys || !d_rows))) return fail(ctx, AM_ERR_INVALID_ARG, "bad arguments");
    if (precision != AM_PREC_FP64 && precision != AM_PREC_MIXED && precision != AM_PREC_TENSOR &&
        precision != AM_PREC_SLICED)
        return fail(ctx, AM_ERR_INVALID_ARG, "unknown precision %d", (int)precision);
    const NetHost &nh = ctx->nets[net_id];
    if (precision == AM_PREC_SLICED) {
        if (n == 0) return AM_OK;
        am_status s = sliced_compose(ctx, net_id, reinterpret_cast<const unsigned long long *>(d_keys), n, d_rows);
        if (s != AM_OK) return s;
        if (d_err) CU(cudaMemsetAsync(d_err, 0, sizeof(float) * n * (nh.N + 1), ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        return AM_OK;
    }
    if (precision != AM_PREC_FP64 && nh.dev.fp64_only)
        return fail(ctx, AM_ERR_INVALID_ARG,
                    "a leaky / parametric ReLU net or one with hidden-layer shortcuts composes in AM_PREC_FP64 only");
    if (precision == AM_PREC_TENSOR && !tc_fits(nh.dev.width, nh.dev.L, ctx->opts.max_neurons))
        return fail(ctx, AM_ERR_INVALID_ARG, "AM_PREC_TENSOR needs 2 n_{l-1} (rounded to 16) <= max_neurons + 10");
    if (n == 0) return AM_OK;
    MarchArgs ma{};
    ma.nets = ctx->d_nets;
    ma.ar = ctx->ar;
    ma.max_n = ctx->opts.max_neurons;
    ma.max_w = ctx->opts.max_width;
    ma.tc = precision == AM_PREC_TENSOR ? 1 : 0;
    launch_compose(ma, precision == AM_PREC_FP64 ? 0 : 1, ctx->d_nets + net_id,
                   reinterpret_cast<const unsigned long long *>(d_keys), nh.dev.kw, n, d_rows, d_err, ctx->stream);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->stats.kernel_launches += 1;
    return AM_OK;
}

am_status am_compose_neighbors(am_ctx *ctx, int net_id, const uint64_t *d_parent_keys, const double *d_parent_rows,
                               const int32_t *d_flip, int64_t n, double *d_rows)
{
    if (!ctx || !ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "no context");
    if (net_id < 0 || net_id >= (int)ctx->nets.size()) return fail(ctx, AM_ERR_INVALID_ARG, "unknown net %d", net_id);
    if (n < 0 || (n > 0 && (!d_parent_keys || !d_parent_rows || !d_flip || !d_rows)))
        return fail(ctx, AM_ERR_INVALID_ARG, "bad arguments");
    const NetHost &nh = ctx->nets[net_id];
    if (!nh.oz_ok) return fail(ctx, AM_ERR_INVALID_ARG, "the rank-1 compose needs every hidden fan-in <= %d", kOzMaxFanIn);
    if (n == 0) return AM_OK;
    if (n > (int64_t)1 << 26) return fail(ctx, AM_ERR_CAPACITY, "at most 2^26 neighbours per call");
    am_status s = ensure_oz_scratch(ctx);
    if (s == AM_OK) s = ensure_r1_scratch(ctx);
    if (s != AM_OK) return s;
    const int N = nh.dev.N, L = nh.dev.L, kw = nh.dev.kw;
    // host: the flips (checked), each child's key, the order by flip layer
    std::vector<int32_t> flip(n);
    std::vector<unsigned long long> keys((size_t)n * kw);
    CU(cudaMemcpy(flip.data(), d_flip, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(keys.data(), d_parent_keys, sizeof(unsigned long long) * n * kw, cudaMemcpyDeviceToHost));
    std::vector<int> layer(n);
    int64_t cnt[kMaxLayers + 2] = {};
    for (int64_t i = 0; i < n; ++i) {
        const int e = flip[i];
        if (e < 0 || e >= N) return fail(ctx, AM_ERR_INVALID_ARG, "flip %d of item %lld is not a neuron", e, (long long)i);
        int l = L;
        for (int ll = 1; ll <= L; ++ll)
            if (e < nh.dev.row0[ll] + nh.dev.width[ll]) { l = ll; break; }
        layer[i] = l;
        cnt[l] += 1;
        keys[(size_t)i * kw + (e >> 6)] ^= 1ull << (e & 63);
    }
    std::vector<int32_t> order(n), ident(n);
    for (int64_t i = 0; i < n; ++i) ident[i] = (int32_t)i;
    int64_t cnt_le[kMaxLayers + 1] = {}, pos[kMaxLayers + 2] = {};
    for (int l = 1; l <= L; ++l) {
        cnt_le[l] = cnt_le[l - 1] + cnt[l];
        pos[l] = cnt_le[l - 1];
    }
    for (int64_t i = 0; i < n; ++i) order[pos[layer[i]]++] = (int32_t)i;
    // device: keys, identity parents, flips, the order, the rows as FP32 pairs (in and out)
    const int64_t rstride = 8 * (int64_t)(N + 1);
    unsigned long long *dk = nullptr;
    int32_t *dpar = nullptr, *dflip = nullptr, *dord = nullptr;
    float *pin = nullptr, *pout = nullptr;
    am_status rc = AM_OK;
    auto release = [&]() {
        for (void *b : {(void *)dk, (void *)dpar, (void *)dflip, (void *)dord, (void *)pin, (void *)pout})
            if (b) cudaFree(b);
    };
    cudaError_t e = cudaSuccess;
    if (!e) e = cudaMalloc(&dk, sizeof(unsigned long long) * n * kw);
    if (!e) e = cudaMalloc(&dpar, sizeof(int32_t) * n);
    if (!e) e = cudaMalloc(&dflip, sizeof(int32_t) * n);
    if (!e) e = cudaMalloc(&dord, sizeof(int32_t) * n);
    if (!e) e = cudaMalloc(&pin, sizeof(float) * rstride * n);
    if (!e) e = cudaMalloc(&pout, sizeof(float) * rstride * n);
    if (!e) e = cudaMemcpyAsync(dk, keys.data(), sizeof(unsigned long long) * n * kw, cudaMemcpyHostToDevice, ctx->stream);
    if (!e) e = cudaMemcpyAsync(dpar, ident.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (!e) e = cudaMemcpyAsync(dflip, flip.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (!e) e = cudaMemcpyAsync(dord, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (!e) {
        rows_to_pairs(d_parent_rows, pin, n, N + 1, ctx->stream);
        e = cudaGetLastError();
    }
    if (!e) {
        const R1Cells cells{dk, kw, dpar, dflip};
        e = oz_rank1(oz_view(nh), cells, dord, n, cnt_le, pin, 0, pout, 0, ctx->oz, ctx->r1, ctx->oz_tile_cells,
                     ctx->sm_count, ctx->stream);
    }
    if (!e) {
        pairs_to_rows(pout, d_rows, n, N + 1, ctx->stream);
        e = cudaGetLastError();
    }
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    release();
    if (e) return fail(ctx, AM_ERR_CUDA, "am_compose_neighbors: %s", cudaGetErrorString(e));
    rc = sliced_check(ctx);
    return rc;
}

am_status am_set_tuning(am_ctx *ctx, const am_tuning *t)
{
    if (!ctx || !ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "no context");
    if (!t) return fail(ctx, AM_ERR_INVALID_ARG, "null tuning");
    int nt = 0;
    const int *tc = oz_tile_cells(&nt);
    bool ok = t->compose_tile_cells == 0;
    for (int i = 0; i < nt; ++i) ok = ok || t->compose_tile_cells == tc[i];
    if (!ok) return fail(ctx, AM_ERR_INVALID_ARG, "unsupported compose_tile_cells %d", t->compose_tile_cells);
    if (t->rank1_period < 0 || t->rank1_period > 1 << 20)
        return fail(ctx, AM_ERR_INVALID_ARG, "rank1_period %d out of range", t->rank1_period);
    if (t->clip_kernel != 0 && t->clip_kernel != 1)
        return fail(ctx, AM_ERR_INVALID_ARG, "clip_kernel %d: 0 or 1", t->clip_kernel);
    if (t->check_kernel != 0 && t->check_kernel != 1)
        return fail(ctx, AM_ERR_INVALID_ARG, "check_kernel %d: 0 or 1", t->check_kernel);
    ctx->oz_tile_cells = t->compose_tile_cells;
    ctx->oz_rank1_period = t->rank1_period;
    ctx->clip_kernel = t->clip_kernel;
    ctx->check_kernel = t->check_kernel;
    return AM_OK;
}

am_status am_get_tuning(const am_ctx *ctx, am_tuning *t)
{
    if (!ctx || !t) return AM_ERR_INVALID_ARG;
    t->compose_tile_cells = ctx->oz_tile_cells;
    t->rank1_period = ctx->oz_rank1_period;
    t->clip_kernel = ctx->clip_kernel;
    t->check_kernel = ctx->check_kernel;
    return AM_OK;
}

am_status am_autotune_compose(am_ctx *ctx, int net_id, const uint64_t *d_keys, int64_t n, double *d_rows, int reps,
                              am_tune_point *h_points, int max_points, int *n_points)
{
    if (!ctx || !ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "no context");
    if (net_id < 0 || net_id >= (int)ctx->nets.size()) return fail(ctx, AM_ERR_INVALID_ARG, "unknown net %d", net_id);
    if (n < 1 || !d_keys || !d_rows || reps < 1 || max_points < 0 || (max_points > 0 && !h_points))
        return fail(ctx, AM_ERR_INVALID_ARG, "bad arguments");
    const auto *keys = reinterpret_cast<const unsigned long long *>(d_keys);
    int nt = 0;
    const int *tiles = oz_tile_cells(&nt);
    const int saved = ctx->oz_tile_cells;
    int best = -1;
    float best_ms = 0.0f;
    for (int i = 0; i < nt; ++i) {
        ctx->oz_tile_cells = tiles[i];
        am_status s = sliced_compose(ctx, net_id, keys, n, d_rows);     // warm-up, untimed
        if (s != AM_OK) { ctx->oz_tile_cells = saved; return s; }
        std::vector<float> ms(reps);
        for (int r = 0; r < reps; ++r) {
            CU(cudaEventRecord(ctx->evk0, ctx->stream));
            s = sliced_compose_async(ctx, net_id, keys, ctx->nets[net_id].dev.kw, n, d_rows);
            if (s != AM_OK) { ctx->oz_tile_cells = saved; return s; }
            CU(cudaEventRecord(ctx->evk1, ctx->stream));
            CU(cudaEventSynchronize(ctx->evk1));
            CU(cudaEventElapsedTime(&ms[r], ctx->evk0, ctx->evk1));
        }
        s = sliced_check(ctx);
        if (s != AM_OK) { ctx->oz_tile_cells = saved; return s; }
        std::sort(ms.begin(), ms.end());
        const float med = ms[reps / 2];
        if (i < max_points) {
            h_points[i].compose_tile_cells = tiles[i];
            h_points[i].ms = med;
        }
        // a later candidate must win by more than 1 % (timing noise): ties keep the earlier one,
        // and the automatic choice, which adapts to every batch size, comes first
        if (best < 0 || med < best_ms * 0.99f) { best = tiles[i]; best_ms = med; }
    }
    ctx->oz_tile_cells = best;
    if (n_points) *n_points = nt;
    return AM_OK;
}

am_status am_autotune_march(am_ctx *ctx, int net_id, const double *h_origins, const double *h_dirs, int n_rays,
                            double R, int64_t max_cells, int reps, am_march_opts *best, am_march_point *h_points,
                            int max_points, int *n_points)
{
    if (!ctx || !ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "no context");
    if (net_id < 0 || net_id >= (int)ctx->nets.size()) return fail(ctx, AM_ERR_INVALID_ARG, "unknown net %d", net_id);
    if (!best || reps < 1 || max_cells < 0 || max_points < 0 || (max_points > 0 && !h_points))
        return fail(ctx, AM_ERR_INVALID_ARG, "bad arguments");
    struct Cand { am_precision p; am_schedule s; };
    std::vector<Cand> cands = {{AM_PREC_FP64, AM_SCHED_PERSISTENT}, {AM_PREC_MIXED, AM_SCHED_PERSISTENT},
                               {AM_PREC_FP64, AM_SCHED_LEVELS}, {AM_PREC_MIXED, AM_SCHED_LEVELS}};
    if (ctx->nets.size() == 1 && ctx->nets[0].oz_ok) cands.push_back({AM_PREC_SLICED, AM_SCHED_LEVELS});
    int bi = -1;
    float bms = 0.0f;
    for (size_t c = 0; c < cands.size(); ++c) {
        am_march_opts op = *best;
        op.precision = cands[c].p;
        op.schedule = cands[c].s;
        op.max_cells = max_cells;
        std::vector<float> ms;
        for (int r = 0; r <= reps; ++r) {                  // run 0 warms up
            am_status s = am_reset(ctx);
            if (s == AM_OK) s = am_seed(ctx, net_id, h_origins, h_dirs, n_rays, R, nullptr);
            if (s == AM_OK) s = am_march(ctx, &op);
            if (s != AM_OK && s != AM_INCOMPLETE) return s;
            if (r > 0) ms.push_back((float)ctx->stats.ms_march);
        }
        std::sort(ms.begin(), ms.end());
        const float med = ms[ms.size() / 2];
        if ((int)c < max_points) h_points[c] = am_march_point{cands[c].p, cands[c].s, med};
        if (bi < 0 || med < bms) { bi = (int)c; bms = med; }
    }
    am_status s = am_reset(ctx);
    if (s != AM_OK) return s;
    best->precision = cands[bi].p;
    best->schedule = cands[bi].s;
    if (n_points) *n_points = (int)cands.size();
    return AM_OK;
}

am_status am_proposal_samples(am_ctx *ctx, int net_id, float *d_X, float *d_Y, int64_t max_samples,
                              int64_t *n_samples)
{
    if (!ctx || !ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "no context");
    if (!ctx->mesh_valid || net_id < 0 || net_id >= (int)ctx->mesh.size())
        return fail(ctx, AM_ERR_STATE, "no mesh for net %d: call am_march", net_id);
    if (!n_samples || max_samples < 0) return fail(ctx, AM_ERR_INVALID_ARG, "bad arguments");
    const MeshInfo &mi = ctx->mesh[net_id];
    const int64_t n = std::min(mi.corners, max_samples);
    *n_samples = n;
    if (!d_X || !d_Y || n == 0) return AM_OK;
    const NetHost &nh = ctx->nets[net_id];
    SampleArgs a{};
    a.ar = ctx->ar;
    a.perm = ctx->d_perm;
    a.coff = ctx->d_coff;
    a.f0 = mi.face_base;
    a.nf = mi.faces;
    a.c0 = mi.corner_base;
    a.max_samples = n;
    a.N = nh.dev.N;
    a.L = nh.dev.L;
    a.n_in = 7 + nh.dev.L;
    for (int l = 0; l <= nh.dev.L; ++l) { a.row0[l] = nh.dev.row0[l]; a.width[l] = nh.dev.width[l]; }
    a.X = d_X;
    a.Y = d_Y;
    launch_proposal_samples(a, ctx->stream);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->stats.kernel_launches += 1;
    return AM_OK;
}

am_status am_proposal_init(am_ctx *ctx, int n_in, int hidden, int n_out, int max_batch, uint64_t seed)
{
    if (!ctx || !ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "no context");
    if (n_in < 1 || n_in > 64 || hidden < 2 || hidden > 768 || (hidden & 1) || n_out < 1 || n_out > kMaxNeurons ||
        max_batch < 1)
        return fail(ctx, AM_ERR_INVALID_ARG, "proposal shape out of range (n_in <= 64, even hidden <= 768)");
    proposal_free(ctx->prop);
    CU(proposal_alloc(ctx->prop, n_in, hidden, n_out, max_batch));
    ProposalDev &p = ctx->prop;
    // Kaiming-normal weights (Box-Muller on splitmix64 draws), zero biases, output bias logit(1/32)
    std::vector<float> w((size_t)p.n_params, 0.0f);
    unsigned long long st = seed * 0x9E3779B97F4A7C15ull + 0x5EEDull;
    auto normal = [&]() {
        const double u1 = ((splitmix64(st++) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((splitmix64(st++) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    };
    const int fans[3] = {n_in, hidden, hidden};
    const double gains[3] = {2.0, 2.0, 1.0};
    for (int l = 0; l < 3; ++l) {
        const double sd = sqrt(gains[l] / fans[l]);
        for (int64_t i = p.off[2 * l]; i < p.off[2 * l + 1]; ++i) w[i] = (float)(sd * normal());
    }
    for (int64_t i = p.off[5]; i < p.off[6]; ++i) w[i] = (float)log(1.0 / 31.0);
    CU(cudaMemcpyAsync(p.w, w.data(), sizeof(float) * p.n_params, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemsetAsync(p.m, 0, sizeof(float) * p.n_params, ctx->stream));
    CU(cudaMemsetAsync(p.v, 0, sizeof(float) * p.n_params, ctx->stream));
    proposal_sync_copies(p, ctx->stream);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(ctx->stream));
    return AM_OK;
}

am_status am_proposal_get_params(am_ctx *ctx, float *h, int64_t n)
{
    if (!ctx || !ctx->prop.w) return fail(ctx, AM_ERR_STATE, "no proposal");
    if (!h || n != ctx->prop.n_params) return fail(ctx, AM_ERR_INVALID_ARG, "expected %lld parameters",
                                                   (long long)ctx->prop.n_params);
    CU(cudaMemcpyAsync(h, ctx->prop.w, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return AM_OK;
}

am_status am_proposal_set_params(am_ctx *ctx, const float *h, int64_t n)
{
    if (!ctx || !ctx->prop.w) return fail(ctx, AM_ERR_STATE, "no proposal");
    if (!h || n != ctx->prop.n_params) return fail(ctx, AM_ERR_INVALID_ARG, "expected %lld parameters",
                                                   (long long)ctx->prop.n_params);
    CU(cudaMemcpyAsync(ctx->prop.w, h, sizeof(float) * n, cudaMemcpyHostToDevice, ctx->stream));
    proposal_sync_copies(ctx->prop, ctx->stream);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(ctx->stream));
    return AM_OK;
}

am_status am_proposal_forward(am_ctx *ctx, const float *d_X, int n, float *d_Z)
{
    if (!ctx || !ctx->prop.w) return fail(ctx, AM_ERR_STATE, "no proposal");
    if (!d_X || !d_Z || n < 1) return fail(ctx, AM_ERR_INVALID_ARG, "bad arguments");
    CU(proposal_forward(ctx->prop, d_X, n, d_Z, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (ctx->prop.tc.ok) {
        int herr = 0;
        CU(cudaMemcpy(&herr, ctx->prop.tc.err, sizeof(int), cudaMemcpyDeviceToHost));
        if (herr) {
            CU(cudaMemset(ctx->prop.tc.err, 0, sizeof(int)));
            return fail(ctx, AM_ERR_TIMEOUT, "a tensor-core pipeline wait of the proposal gave up");
        }
    }
    return AM_OK;
}

am_status am_proposal_grad(am_ctx *ctx, const float *d_X, const float *d_Y, int n, float *h_grads, int64_t n_params,
                           float *h_loss)
{
    if (!ctx || !ctx->prop.w) return fail(ctx, AM_ERR_STATE, "no proposal");
    if (!d_X || !d_Y || !h_grads || !h_loss || n < 1 || n > ctx->prop.max_batch || n_params != ctx->prop.n_params)
        return fail(ctx, AM_ERR_INVALID_ARG, "bad arguments");
    CU(proposal_grad(ctx->prop, d_X, d_Y, n, h_loss, ctx->stream));
    CU(cudaMemcpyAsync(h_grads, ctx->prop.g, sizeof(float) * n_params, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return AM_OK;
}

am_status am_proposal_train(am_ctx *ctx, const float *d_X, const float *d_Y, int64_t n, int batch, int steps,
                            float lr, float *h_losses)
{
    if (!ctx || !ctx->prop.w) return fail(ctx, AM_ERR_STATE, "no proposal");
    if (!d_X || !d_Y || batch < 1 || batch > ctx->prop.max_batch || n < batch || steps < 0 || !(lr > 0.0f))
        return fail(ctx, AM_ERR_INVALID_ARG, "bad training arguments");
    CU(proposal_train(ctx->prop, d_X, d_Y, n, batch, steps, lr, h_losses, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return AM_OK;
}

am_status am_get_mesh(am_ctx *ctx, int net_id, am_mesh *m)
{
    if (!ctx || !m) return fail(ctx, AM_ERR_INVALID_ARG, "null argument");
    if (net_id < 0 || net_id >= (int)ctx->nets.size()) return fail(ctx, AM_ERR_INVALID_ARG, "unknown net %d", net_id);
    if (!ctx->mesh_valid || net_id >= (int)ctx->mesh.size()) return fail(ctx, AM_ERR_STATE, "no mesh: call am_march");
    const MeshInfo &mi = ctx->mesh[net_id];
    m->n_vertices = mi.verts;
    m->n_faces = mi.faces;
    m->n_corners = mi.corners;
    m->key_words = ctx->ar.kw;
    const bool copy = m->xyz || m->face_offsets || m->face_vertices || m->edge_planes || m->face_keys;
    if (!copy) {
        m->n_open_faces = -1;
        return AM_OK;
    }
    if (!m->xyz || !m->face_offsets || !m->face_vertices || !m->edge_planes || !m->face_keys)
        return fail(ctx, AM_ERR_INVALID_ARG, "either all or none of the mesh arrays must be given");
    CU(cudaMemcpyAsync(m->xyz, ctx->d_xyz + 3 * mi.vert_base, sizeof(double) * 3 * mi.verts, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaMemcpyAsync(m->face_vertices, ctx->d_fv + mi.corner_base, sizeof(int32_t) * mi.corners,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(m->edge_planes, ctx->d_fe + mi.corner_base, sizeof(int32_t) * mi.corners,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(m->face_offsets, ctx->d_coff + mi.face_base, sizeof(int64_t) * (mi.faces + 1),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(m->face_keys, ctx->d_fkeys + mi.face_base * ctx->ar.kw,
                       sizeof(unsigned long long) * mi.faces * ctx->ar.kw, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    const int N = ctx->nets[net_id].N;
    int64_t open = 0;
    for (int64_t f = 0; f <= mi.faces; ++f) m->face_offsets[f] -= mi.corner_base;
    for (int64_t f = 0; f < mi.faces; ++f) {
        for (int64_t c = m->face_offsets[f]; c < m->face_offsets[f + 1]; ++c)
            if (m->edge_planes[c] >= N) { ++open; break; }
    }
    m->n_open_faces = open;
    return AM_OK;
}

am_status am_get_mesh_device(am_ctx *ctx, int net_id, am_mesh *m)
{
    if (!ctx || !m) return fail(ctx, AM_ERR_INVALID_ARG, "null argument");
    if (net_id < 0 || net_id >= (int)ctx->nets.size()) return fail(ctx, AM_ERR_INVALID_ARG, "unknown net %d", net_id);
    if (!ctx->mesh_valid || net_id >= (int)ctx->mesh.size()) return fail(ctx, AM_ERR_STATE, "no mesh: call am_march");
    const MeshInfo &mi = ctx->mesh[net_id];
    // every net's rebased offsets get their own region: face_base + net_id, faces + 1 long
    int64_t total = 0;
    for (const MeshInfo &x : ctx->mesh) total += x.faces + 1;
    CU(grow(&ctx->d_coff_net, &ctx->coff_net_cap, total));
    int64_t *off = ctx->d_coff_net + mi.face_base + net_id;
    launch_rebase_offsets(ctx->d_coff + mi.face_base, mi.corner_base, off, mi.faces + 1, ctx->stream);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->stats.kernel_launches += 1;
    m->n_vertices = mi.verts;
    m->n_faces = mi.faces;
    m->n_corners = mi.corners;
    m->key_words = ctx->ar.kw;
    m->n_open_faces = -1;
    m->xyz = ctx->d_xyz + 3 * mi.vert_base;
    m->face_offsets = off;
    m->face_vertices = ctx->d_fv + mi.corner_base;
    m->edge_planes = ctx->d_fe + mi.corner_base;
    m->face_keys = reinterpret_cast<uint64_t *>(ctx->d_fkeys + mi.face_base * ctx->ar.kw);
    return AM_OK;
}

am_status am_test_stall_next_march(am_ctx *ctx, int64_t unpublished_ids, double wait_limit_ms)
{
    if (!ctx || !ctx->ar.keys) return fail(ctx, AM_ERR_STATE, "no context");
    if (!(wait_limit_ms > 0.0 && wait_limit_ms <= 4000.0))
        return fail(ctx, AM_ERR_INVALID_ARG, "wait_limit_ms must lie in (0, 4000]");
    if (unpublished_ids < 1 || unpublished_ids > ctx->ar.cap)
        return fail(ctx, AM_ERR_INVALID_ARG, "unpublished_ids must lie in [1, max_cells]");
    ctx->test_stall_ids = unpublished_ids;
    ctx->test_wait_ns = (long long)(wait_limit_ms * 1e6);
    return AM_OK;
}

am_status am_get_stats(const am_ctx *ctx, am_stats_t *s)
{
    if (!ctx || !s) return AM_ERR_INVALID_ARG;
    *s = ctx->stats;
    return AM_OK;
}

}  // extern "C"
