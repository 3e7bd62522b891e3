// C ABI of the solver (include/fermi.h) and the host orchestration of the method.
//
// Every call runs on a plan: the instances of the call (one for fo_density_matrix, many for
// fo_density_matrix_batched), sorted by size, with their workspace layout, the
// block-to-instance prefix sums of every grouped launch, one tensor map per bucket of
// equally sized instances and the tile width chosen by the autotuner. Plans are cached per
// context (keyed by sizes and parameters); a call writes its per-instance inputs with one
// small kernel and enqueues one launch per stage for the whole batch, optionally replayed
// as a CUDA graph. The host only plans, checks arguments and enqueues kernels: every number
// of the method is computed on the device, and nothing synchronises until the optional
// readback of the scalar results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace fo;

namespace {

enum PlanMode { MODE_DENSITY = 0, MODE_MOMENTS = 1, MODE_PRODUCT = 2, MODE_BOUNDS = 3, MODE_COEFFS = 4 };

struct PlanKey {
    std::vector<int64_t> n;
    int mode = MODE_DENSITY, n_terms = 1, k_req = 0, prec = 0, mu_mode = 0, n_quad = 0;
    int use_given = 0, tile_req = 0, ctas_req = 0, drain_req = 0, store_req = 0, sym = 1, max_bisect = 0, max_newton = 0, staged = 0, lanczos = 0, power = 0, nofix = 0;
    int chain = 0, chain_win = 0, persist_req = 0;
    double tr_tol = 0.0;
    bool operator==(const PlanKey& o) const {
        return n == o.n && mode == o.mode && n_terms == o.n_terms && k_req == o.k_req && prec == o.prec &&
               mu_mode == o.mu_mode && n_quad == o.n_quad && use_given == o.use_given &&
               tile_req == o.tile_req && ctas_req == o.ctas_req && drain_req == o.drain_req &&
               store_req == o.store_req && sym == o.sym && max_bisect == o.max_bisect &&
               max_newton == o.max_newton && tr_tol == o.tr_tol && staged == o.staged && lanczos == o.lanczos && power == o.power &&
               nofix == o.nofix && chain == o.chain && chain_win == o.chain_win && persist_req == o.persist_req;
    }
};

struct Bucket {
    int64_t np;
    int first, count;
    size_t off;           // workspace offset of the bucket's slot region
    int64_t inst_bytes;   // slot region of one instance
};

struct Group {           // instances [i0, i1) with buckets [b0, b0 + nb): one grouped launch
    int i0, i1, b0, nb;
};

struct HostWork {
    std::vector<int> pre;
    Work dev{nullptr, 0, 0};
};

struct Plan {
    PlanKey key;
    uint64_t ws_gen = 0;
    int batch = 0;
    Shape sh{};
    bool giants = false, moments = false;
    bool fix = false;         // split forms with mu searched: trace correction after the expansion
    int chain = 0;            // split forms: each chain of products (baby, giant, Clenshaw) in one launch
    int chain_win = 0;        // tiles per step of a chain launch's instance windows (0: one window)
    int* counters = nullptr;  // chain launches: ticket and per-instance tile counters (workspace)
    int n_slots = 0;
    std::vector<int> order;   // sorted position -> caller index
    std::vector<Inst> inst;   // host copy, sorted
    std::vector<Bucket> buckets;
    std::vector<Group> groups;
    std::vector<unsigned char> maps;   // 256 bytes per bucket: K-major and MN-major tensor maps
    std::vector<GramBucket> gram_bk;   // float32 master geometry of the Frobenius-product kernel
    std::vector<GramGroup> gram_grp;
    GramGeom gram_geom{};
    HostWork wg, wsc, we, wr, wgr, wct, wtc[2], wf64;   // wtc[0]: 256-wide tiles, wtc[1]: 128-wide
    int tile_n = 0;
    int tile_ctas = 0;
    int tile_drain = 0;
    int tile_store = 0;   // 1: full planes, 2: upper 128-blocks (sh.ublk); 0 for FP64
    int tile_persist = 0; // 1: the persistent kernel (128-wide tiles, separate epilogue warps)
    int npairs = 0;
    void* dtab = nullptr;     // device tables: Inst[], InstIO[], prefixes
    Inst* d_inst = nullptr;
    InstIO* d_io = nullptr;
    DevResult* d_res = nullptr;   // batch results, sorted order (in the workspace)
    double* ct = nullptr;
    double* part_g = nullptr;
    double* part_t = nullptr;
    double* part_tc = nullptr;    // per-tile (tr, ||.||^2) partials of the float64-output products
    float* lscratch = nullptr;    // learned mu: features, normalised features, activations, outputs
    int* lcount = nullptr;        // learned mu: instances still active after a judge
    size_t total = 0;
    double flops_product = 0.0;   // algorithmic flops of one product over the batch
    cudaGraphExec_t graph = nullptr;
    int graph_launches = 0;   // kernels in the captured graph
    ~Plan() {
        if (graph) cudaGraphExecDestroy(graph);
        if (dtab) cudaFree(dtab);
    }
};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

struct ProfEntry {
    cudaEvent_t a, b;
    int stage;
    double flops;
    int launches;
};

struct fo_ctx {
    int device = 0;
    bool prof = false;
    std::vector<ProfEntry> prof_pending;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[FO_PROFILE_STAGES] = {0};
    double prof_flops[FO_PROFILE_STAGES] = {0};
    int64_t prof_launches[FO_PROFILE_STAGES] = {0};
    int64_t prof_calls = 0;
    int num_sms = 0;
    std::string err;
    void* ws = nullptr;        // device workspace shared by the plans
    size_t ws_bytes = 0;
    uint64_t ws_gen = 1;       // bumped when the workspace moves (cached plans go stale)
    // host-buffer entry point: two device staging slots used in turn, copy streams
    struct HostSlot {
        void* buf = nullptr;
        size_t bytes = 0;
        cudaEvent_t in = nullptr, done = nullptr, out = nullptr;   // inputs copied, solved, outputs copied
        bool used = false;
    };
    HostSlot hslot[2];
    int hnext = 0;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    int* flag = nullptr;       // [0] tensor-core wait timeout, [1..3] self-check record
    std::vector<std::unique_ptr<Plan>> plans;   // most recently used last
    DevResult* hres = nullptr; // pinned readback buffer
    size_t hres_count = 0;
    cudaStream_t cap = nullptr;   // stream for graph capture
    bool capturing = false;
    int* hcount = nullptr;        // pinned readback of the learned judge's active count
    // learned-mu model (device, float32): parameters, gradients, Adam moments, normalisation
    float* mlp = nullptr;         // params | grad | m | v | norm
    bool mlp_ready = false;       // trained, loaded or set
    int mlp_step = 0;             // Adam steps taken
    float* mlp_scratch = nullptr; // training buffers
    size_t mlp_scratch_floats = 0;
};

namespace {

constexpr size_t kMaxPlans = 8;
// Learned expansion order: the network's proposed order is enlarged by this factor (then
// rounded up to whole giant steps) before it cuts the expansion.
constexpr double kOrderMargin = 1.25;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

fo_status fail(fo_ctx* ctx, fo_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return st;
}

fo_status cuda_fail(fo_ctx* ctx, cudaError_t e, const char* where) {
    return fail(ctx, FO_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// FERMI_DEBUG_SYNC=1: synchronise after every enqueued stage so that an asynchronous
// device error is attributed to the stage that raised it.
bool debug_sync() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("FERMI_DEBUG_SYNC");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v == 1;
}

// FERMI_AUTOTUNE_LOG=1: print every autotuned plan's candidate timings to stderr.
bool autotune_log() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("FERMI_AUTOTUNE_LOG");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v == 1;
}

#define FO_CUDA(call, where)                                                              \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ == cudaSuccess && debug_sync() && !ctx->capturing) e_ = cudaDeviceSynchronize(); \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where);                          \
    } while (0)

#define FO_TRY(x)                      \
    do {                               \
        fo_status s_ = (x);            \
        if (s_ != FO_OK) return s_;    \
    } while (0)

// ---------------------------------------------------------------- stage profiler
cudaEvent_t ev_get(fo_ctx* ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Starts a timed stage when profiling is on (and not capturing); returns a handle or -1.
int prof_begin(fo_ctx* ctx, cudaStream_t st, int stage) {
    if (!ctx->prof || ctx->capturing) return -1;
    ProfEntry e{ev_get(ctx), ev_get(ctx), stage, 0.0, 0};
    cudaEventRecord(e.a, st);
    ctx->prof_pending.push_back(e);
    return (int)ctx->prof_pending.size() - 1;
}

void prof_end(fo_ctx* ctx, cudaStream_t st, int h, double flops, int launches) {
    if (h < 0) return;
    ProfEntry& e = ctx->prof_pending[h];
    e.flops = flops;
    e.launches = launches;
    cudaEventRecord(e.b, st);
}

void prof_collect(fo_ctx* ctx) {
    for (ProfEntry& e : ctx->prof_pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(e.b) == cudaSuccess && cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
            ctx->prof_ms[e.stage] += ms;
            ctx->prof_flops[e.stage] += e.flops;
            ctx->prof_launches[e.stage] += e.launches;
        }
        ctx->ev_pool.push_back(e.a);
        ctx->ev_pool.push_back(e.b);
    }
    ctx->prof_pending.clear();
}

void drop_plans(fo_ctx* ctx) {
    if (ctx->plans.empty()) return;
    cudaDeviceSynchronize();
    ctx->plans.clear();
}

fo_status ensure_ws(fo_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return FO_OK;
    drop_plans(ctx);
    if (ctx->ws) {
        cudaDeviceSynchronize();
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    ctx->ws_gen += 1;
    if (cudaMalloc(&ctx->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, FO_ERR_NOMEM, "workspace allocation of " + std::to_string(bytes) + " bytes failed");
    }
    if (cudaMemset(ctx->ws, 0, bytes) != cudaSuccess) return fail(ctx, FO_ERR_CUDA, "workspace clear failed");
    ctx->ws_bytes = bytes;
    return FO_OK;
}

// --------------------------------------------------------------------------- plan
bool plan_km(int n_terms, int k_req, int* k, int* m) {
    if (n_terms < 1) return false;
    int kk = k_req > 0 ? k_req : (int)std::ceil(std::sqrt((double)n_terms));
    if (kk < 1) kk = 1;
    *k = kk;
    *m = (n_terms + kk - 1) / kk;
    return true;
}

int split_count(int prec) { return prec == FO_PREC_BF16X3 ? 6 : (prec == FO_PREC_FP16X2 ? 3 : 1); }

// Shape, sort order, buckets and the workspace layout (offsets only).
fo_status layout_plan(fo_ctx* ctx, const PlanKey& key, Plan* p) {
    const int batch = (int)key.n.size();
    if (batch < 1) return fail(ctx, FO_ERR_ARG, "batch must be >= 1");
    for (int64_t n : key.n) {
        if (n < 1) return fail(ctx, FO_ERR_ARG, "n must be >= 1");
        if (n > 65536) return fail(ctx, FO_ERR_ARG, "n above 65536 is not supported");
    }
    if (key.n_terms < 1 || key.n_terms > 4096) return fail(ctx, FO_ERR_ARG, "n_terms must be in [1, 4096]");
    if (key.prec < FO_PREC_FP64 || key.prec > FO_PREC_BF16X1) return fail(ctx, FO_ERR_ARG, "unknown precision");
    if (key.tile_req != 0 && key.tile_req != 128 && key.tile_req != 256)
        return fail(ctx, FO_ERR_ARG, "tile_n must be 0, 128 or 256");
    p->key = key;
    p->batch = batch;
    Shape& sh = p->sh;
    std::memset(&sh, 0, sizeof(sh));
    sh.n_terms = key.n_terms;
    if (!plan_km(key.n_terms, key.k_req, &sh.k, &sh.m)) return fail(ctx, FO_ERR_ARG, "bad k");
    if (sh.k > 64 || sh.m > 64) return fail(ctx, FO_ERR_ARG, "k and m must not exceed 64");
    sh.km = sh.k * sh.m;
    sh.M = key.n_quad > 0 ? key.n_quad : std::max(2048, 4 * key.n_terms);
    if (sh.M < key.n_terms) return fail(ctx, FO_ERR_ARG, "n_quad must be >= n_terms");
    sh.is64 = key.prec == FO_PREC_FP64;
    sh.planes = tc_planes(key.prec);
    sh.fp16 = key.prec == FO_PREC_FP16X2;
    // fp16 planes hold v * scale; T slots have |entries| <= 1 (spectrum of X in [-1, 1])
    sh.pscale_t = 256.0f;
    sh.pscale_r = 1.0f;
    const bool bisect = key.mode == MODE_DENSITY && key.mu_mode == FO_MU_BISECT;
    const bool learned = key.mode == MODE_DENSITY && (key.mu_mode == FO_MU_LEARNED || key.mu_mode == FO_MU_ORDER);
    p->giants = (bisect || learned) && sh.m > 2;   // the learned mode falls back to exact moments
    p->moments = bisect || learned || key.mode == MODE_MOMENTS;
    p->fix = (bisect || learned) && !sh.is64 && sh.m > 1 && !key.nofix;
    p->chain = !sh.is64 && key.mode == MODE_DENSITY && key.chain == 2 ? 1 : 0;
    p->chain_win = key.chain_win;
    if (p->moments && sh.k > 33) return fail(ctx, FO_ERR_UNSUPPORTED, "exact moments support k <= 33");
    if (learned && sh.k > 32) return fail(ctx, FO_ERR_UNSUPPORTED, "learned mu supports k <= 32");
    switch (key.mode) {
        case MODE_DENSITY:
        case MODE_MOMENTS:
            sh.n_tslots = sh.k + (p->giants ? sh.m - 2 : 0);
            p->n_slots = sh.n_tslots + sh.m;
            break;
        case MODE_PRODUCT:
            sh.n_tslots = 5;   // A, B, C, D, out
            p->n_slots = 5;
            break;
        default:
            sh.n_tslots = 0;
            p->n_slots = 0;
    }
    p->npairs = std::max(1, std::max((sh.m > 1 ? sh.m - 1 : 1) * std::max(1, sh.k - 1), sh.k));

    // sort by padded size (largest first): the longest tiles of a grouped launch start first
    p->order.resize(batch);
    std::iota(p->order.begin(), p->order.end(), 0);
    std::vector<int64_t> npad(batch);
    for (int b = 0; b < batch; ++b) npad[b] = ((key.n[b] + kPad - 1) / kPad) * kPad;
    std::stable_sort(p->order.begin(), p->order.end(), [&](int a, int b) { return npad[a] > npad[b]; });

    // slot regions, bucket by bucket
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += align256(b); return o; };
    p->inst.assign(batch, Inst{});
    for (int j = 0; j < batch; ++j) {
        const int b = p->order[j];
        const int64_t np = npad[b];
        Inst& in = p->inst[j];
        std::memset(&in, 0, sizeof(in));
        in.n = key.n[b];
        in.np = np;
        in.user = b;
        const size_t np2 = (size_t)np * (size_t)np;
        in.slot_bytes = (int64_t)(sh.is64 ? align256(np2 * 8) : align256(np2 * 4 + (size_t)sh.planes * np2 * 2));
        if (p->buckets.empty() || p->buckets.back().np != np) {
            Bucket bk{np, j, 0, 0, (int64_t)in.slot_bytes * p->n_slots};
            p->buckets.push_back(bk);
        }
        in.bucket = (int)p->buckets.size() - 1;
        in.in_bucket = p->buckets.back().count++;
    }
    for (Bucket& bk : p->buckets) bk.off = take((size_t)bk.inst_bytes * bk.count);
    // per-instance float64 arrays
    std::vector<size_t> small(batch);
    const int ndiag = sh.n_tslots + 2;
    for (int j = 0; j < batch; ++j) {
        Inst& in = p->inst[j];
        in.gram_blocks = gram_blocks_for(in.np, sh.is64);
        size_t o = off;
        o += align256(8 * (size_t)sh.km);             // c
        o += align256(8 * (size_t)sh.km);             // g
        o += align256(8 * (size_t)(sh.km + 2));       // tau
        o += align256(8 * (size_t)sh.M);              // w
        o += align256(8 * (size_t)sh.M);              // f
        o += align256(8 * (size_t)ndiag);             // diag
        o += align256(8 * (size_t)p->npairs);         // gram
        o += align256(8 * (size_t)p->npairs * in.gram_blocks);   // gram partials
        o += align256(8 * (3 * (size_t)in.np + 2 * kLzMax + 3));  // Lanczos state
        small[j] = off;
        off = o;
    }
    const size_t off_res = take(sizeof(DevResult) * batch);
    // work lists
    auto fill = [&](HostWork& w, auto count) {
        w.pre.assign(batch + 1, 0);
        for (int j = 0; j < batch; ++j) w.pre[j + 1] = w.pre[j] + (int)count(p->inst[j]);
    };
    fill(p->wg, [](const Inst& in) { return (in.n + kGershRows - 1) / kGershRows; });
    fill(p->wsc, [](const Inst& in) { const int64_t t = in.np / 32; return t * (t + 1) / 2; });
    fill(p->we, [](const Inst& in) { return (int64_t)ew_blocks(in.np); });
    fill(p->wr, [](const Inst& in) { return (int64_t)red_blocks(in.np); });
    fill(p->wgr, [](const Inst& in) { return (int64_t)in.gram_blocks; });
    fill(p->wct, [&](const Inst& in) { return (int64_t)ct_blocks(in.np, sh.k); });
    const bool full = key.mode == MODE_PRODUCT && !key.sym;
    fill(p->wtc[0], [&](const Inst& in) { return full ? tc_tiles_full(in.np, 256) : tc_tiles(in.np, 256); });
    fill(p->wtc[1], [&](const Inst& in) { return full ? tc_tiles_full(in.np, 128) : tc_tiles(in.np, 128); });
    fill(p->wf64, [](const Inst& in) { return f64_tiles(in.np); });
    const size_t off_pg = take(8 * 3 * (size_t)std::max(1, p->wg.pre[batch]));
    const size_t off_pt = take(8 * 2 * (size_t)std::max(1, p->wr.pre[batch]));
    const size_t off_ptc = take(8 * 2 * (size_t)std::max(1, p->wtc[1].pre[batch]));   // 128-blocks
    const size_t off_cnt = take(4 * ((size_t)batch + 8));
    const size_t off_ls = take(4 * (size_t)batch * (2 * kMlpIn + 4 * kMlpHidden + kMlpOut));
    const size_t off_lc = take(sizeof(int));
    p->total = off;
    // remember the offsets in the (not yet placed) pointers
    for (int j = 0; j < batch; ++j) p->inst[j].c = reinterpret_cast<double*>(small[j]);
    p->d_res = reinterpret_cast<DevResult*>(off_res);
    p->part_g = reinterpret_cast<double*>(off_pg);
    p->part_t = reinterpret_cast<double*>(off_pt);
    p->part_tc = reinterpret_cast<double*>(off_ptc);
    p->counters = reinterpret_cast<int*>(off_cnt);
    p->lscratch = reinterpret_cast<float*>(off_ls);
    p->lcount = reinterpret_cast<int*>(off_lc);
    // launch groups: at most kMaxBuckets tensor maps per launch
    for (int b0 = 0; b0 < (int)p->buckets.size(); b0 += kMaxBuckets) {
        const int nb = std::min<int>(kMaxBuckets, (int)p->buckets.size() - b0);
        Group g;
        g.b0 = b0;
        g.nb = nb;
        g.i0 = p->buckets[b0].first;
        const Bucket& last = p->buckets[b0 + nb - 1];
        g.i1 = last.first + last.count;
        p->groups.push_back(g);
    }
    const int s = split_count(key.prec);
    p->flops_product = 0.0;
    for (const Inst& in : p->inst) p->flops_product += (double)s * in.n * in.n * (in.n + 1.0);
    return FO_OK;
}

// Places the plan in the workspace, uploads its tables and builds its tensor maps.
fo_status place_plan(fo_ctx* ctx, Plan* p) {
    char* W = reinterpret_cast<char*>(ctx->ws);
    const Shape& sh = p->sh;
    const int batch = p->batch;
    const int ndiag = sh.n_tslots + 2;
    p->d_res = reinterpret_cast<DevResult*>(W + reinterpret_cast<size_t>(p->d_res));
    p->part_g = reinterpret_cast<double*>(W + reinterpret_cast<size_t>(p->part_g));
    p->part_t = reinterpret_cast<double*>(W + reinterpret_cast<size_t>(p->part_t));
    p->part_tc = reinterpret_cast<double*>(W + reinterpret_cast<size_t>(p->part_tc));
    p->counters = reinterpret_cast<int*>(W + reinterpret_cast<size_t>(p->counters));
    p->lscratch = reinterpret_cast<float*>(W + reinterpret_cast<size_t>(p->lscratch));
    p->lcount = reinterpret_cast<int*>(W + reinterpret_cast<size_t>(p->lcount));
    for (int j = 0; j < batch; ++j) {
        Inst& in = p->inst[j];
        const Bucket& bk = p->buckets[in.bucket];
        in.slots = W + bk.off + (size_t)bk.inst_bytes * in.in_bucket;
        char* o = W + reinterpret_cast<size_t>(in.c);
        auto next = [&](size_t b) { char* r = o; o += align256(b); return reinterpret_cast<double*>(r); };
        in.c = next(8 * (size_t)sh.km);
        in.g = next(8 * (size_t)sh.km);
        in.tau = next(8 * (size_t)(sh.km + 2));
        in.w = next(8 * (size_t)sh.M);
        in.f = next(8 * (size_t)sh.M);
        in.diag = next(8 * (size_t)ndiag);
        in.gram = next(8 * (size_t)p->npairs);
        in.gpart = next(8 * (size_t)p->npairs * in.gram_blocks);
        in.lz = next(8 * (3 * (size_t)in.np + 2 * kLzMax + 3));
        in.res = p->d_res + j;
    }
    // device tables: Inst[batch], InstIO[batch], the prefix arrays, then the cosine table of
    // the coefficient nodes. These stay valid for the plan's life: the workspace is shared
    // by every cached plan of the context, and another plan's call overwrites it.
    HostWork* lists[] = {&p->wg, &p->wsc, &p->we, &p->wr, &p->wgr, &p->wct, &p->wtc[0], &p->wtc[1], &p->wf64};
    size_t bytes = align256(sizeof(Inst) * batch) + align256(sizeof(InstIO) * batch);
    for (HostWork* w : lists) bytes += align256(sizeof(int) * w->pre.size());
    const size_t off_ct = bytes;
    bytes += align256(8 * 4 * (size_t)sh.M);
    if (cudaMalloc(&p->dtab, bytes) != cudaSuccess) {
        cudaGetLastError();
        p->dtab = nullptr;
        return fail(ctx, FO_ERR_NOMEM, "plan table allocation failed");
    }
    std::vector<unsigned char> host(bytes, 0);
    size_t o = 0;
    p->d_inst = reinterpret_cast<Inst*>(reinterpret_cast<char*>(p->dtab) + o);
    std::memcpy(host.data() + o, p->inst.data(), sizeof(Inst) * batch);
    o += align256(sizeof(Inst) * batch);
    p->d_io = reinterpret_cast<InstIO*>(reinterpret_cast<char*>(p->dtab) + o);
    o += align256(sizeof(InstIO) * batch);
    for (HostWork* w : lists) {
        w->dev.pre = reinterpret_cast<const int*>(reinterpret_cast<char*>(p->dtab) + o);
        w->dev.count = batch;
        w->dev.total = w->pre[batch];
        std::memcpy(host.data() + o, w->pre.data(), sizeof(int) * w->pre.size());
        o += align256(sizeof(int) * w->pre.size());
    }
    if (cudaMemcpy(p->dtab, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(ctx, FO_ERR_CUDA, "plan table upload failed");
    p->ct = reinterpret_cast<double*>(reinterpret_cast<char*>(p->dtab) + off_ct);
    // tensor maps: one per bucket over (column, row, plane, slot, instance)
    if (!sh.is64 && p->n_slots > 0) {
        p->maps.assign(256 * p->buckets.size(), 0);
        for (size_t b = 0; b < p->buckets.size(); ++b) {
            const Bucket& bk = p->buckets[b];
            const char* planes0 = W + bk.off + 4 * (size_t)bk.np * (size_t)bk.np;
            std::string err;
            for (int q = 0; q < 2; ++q)   // K-major tiles, then MN-major tiles
                if (!tc_make_map(p->maps.data() + 256 * b + 128 * q, planes0, bk.np, sh.planes, p->n_slots,
                                 bk.count, p->inst[bk.first].slot_bytes, bk.inst_bytes, sh.fp16 != 0, &err,
                                 q == 1))
                    return fail(ctx, FO_ERR_CUDA, "tensor map: " + err);
        }
    }
    // geometry of the float32 masters for the Frobenius products' tensor maps
    if (!sh.is64 && p->n_slots > 0) {
        p->gram_bk.clear();
        for (const Bucket& bk : p->buckets)
            p->gram_bk.push_back(GramBucket{W + bk.off, bk.np, p->inst[bk.first].slot_bytes, bk.inst_bytes, bk.count});
        p->gram_grp.clear();
        for (const Group& g : p->groups) p->gram_grp.push_back(GramGroup{g.b0, g.nb, g.i0, g.i1});
        p->gram_geom = GramGeom{p->gram_bk.data(), p->gram_grp.data(), (int)p->gram_grp.size(), p->n_slots,
                                p->wgr.pre.data()};
    }
    // the cosine table depends on M only (kept in the plan's own device tables)
    cudaError_t e = launch_cos_table(sh.M, p->ct, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cos_table");
    p->ws_gen = ctx->ws_gen;
    return FO_OK;
}

// ---------------------------------------------------------------- products
struct Run {
    int n_gemm = 0;     // products per instance
    int launches = 0;   // kernels launched
};

Step make_step(const Plan& p, int a, int b, int c, int d, int out, double alpha, double beta, double shift,
               bool a_r, bool b_r, bool out_r, bool out64, fo_ctx* ctx) {
    const Shape& sh = p.sh;
    Step st;
    std::memset(&st, 0, sizeof(st));
    st.a = a;
    st.b = b;
    st.c = c;
    st.d = d;
    st.out = out;
    st.out64 = out64 ? 1 : 0;
    st.fp16 = sh.fp16;
    const float sa = sh.fp16 ? (a_r ? sh.pscale_r : sh.pscale_t) : 1.0f;
    const float sb = sh.fp16 ? (b_r ? sh.pscale_r : sh.pscale_t) : 1.0f;
    st.alpha = (float)(alpha / ((double)sa * sb));
    st.beta = (float)beta;
    st.shift = (float)shift;
    st.alpha64 = alpha;
    st.beta64 = beta;
    st.shift64 = shift;
    st.planes = out >= 0 ? sh.planes : 0;
    st.plane_scale = out_r ? sh.pscale_r : sh.pscale_t;
    st.dbg = ctx->flag + 1;
    return st;
}

// Independent products of the whole batch (one stage), at most kMaxSteps per launch.
fo_status run_products(fo_ctx* ctx, Plan& p, const Step* steps, int nsteps, cudaStream_t s, const char* tag,
                       int index, Run* run, int prec = -1) {
    if (prec < 0) prec = p.key.prec;
    // flops of these products: the plan's, scaled to this precision's split products
    const double flops = p.sh.is64 ? p.flops_product : p.flops_product / split_count(p.key.prec) * split_count(prec);
    for (int q0 = 0; q0 < nsteps; q0 += kMaxSteps) {
        const int nq = std::min(kMaxSteps, nsteps - q0);
        const int h = prof_begin(ctx, s, FO_STAGE_PRODUCTS);
        int launches = 0;
        if (p.sh.is64) {
            FO_CUDA(launch_gemm_f64(steps + q0, nq, p.d_inst, p.d_io, p.wf64.dev, s), "gemm_f64");
            launches = 1;
        } else {
            const HostWork& w = p.wtc[p.tile_n == 128 ? 1 : 0];
            for (const Group& g : p.groups) {
                std::string err;
                const int tile0 = w.pre[g.i0];
                cudaError_t e = tc_gemm(prec, p.tile_n, p.tile_ctas, p.tile_drain, steps + q0, nq, p.d_inst, p.d_io,
                                        w.dev.pre, g.i0, g.i1, tile0, w.pre[g.i1] - tile0,
                                        p.maps.data() + 256 * (size_t)g.b0, g.b0, g.nb, ctx->flag, s, &err,
                                        p.key.sym ? (p.sh.ublk ? 2 : 1) : 0, p.tile_persist);
                if (e == cudaSuccess && debug_sync() && !ctx->capturing) e = cudaDeviceSynchronize();
                if (e != cudaSuccess) {
                    const std::string where = std::string("tc_gemm ") + tag + " " + std::to_string(index);
                    if (!err.empty()) return fail(ctx, FO_ERR_CUDA, where + ": " + err);
                    return cuda_fail(ctx, e, where.c_str());
                }
                ++launches;
            }
        }
        prof_end(ctx, s, h, flops * nq, launches);
        run->launches += launches;
        run->n_gemm += nq;
    }
    return FO_OK;
}

fo_status run_product(fo_ctx* ctx, Plan& p, const Step& st, cudaStream_t s, const char* tag, int index,
                      Run* run, int prec = -1) {
    return run_products(ctx, p, &st, 1, s, tag, index, run, prec);
}

// Precision of the trace correction's product P P. Its error enters P only through
// gamma (P - P P) with |gamma| ~ 1e-6 (the correction runs only where it is rounding-sized),
// so BF16x1's ~4e-3 relative error of P P moves P by ~1e-8 at most, far below the 1e-6 bar;
// the plans in BF16x3 form it with one split product instead of six (plane 0 of P). FP16x2
// plans keep their own precision (their planes are scaled float16).
int fix_precision(const Plan& p) { return p.key.prec == FO_PREC_BF16X3 ? FO_PREC_BF16X1 : p.key.prec; }

// A chain of dependent products (step q reads what step q - 1 wrote) of the whole batch: one
// launch per group of instances and per kMaxChain steps when the plan runs chains
// (tc_chain), else one launch per step.
fo_status run_chain(fo_ctx* ctx, Plan& p, const std::vector<Step>& steps, cudaStream_t s, const char* tag,
                    Run* run) {
    if (steps.empty()) return FO_OK;
    if (!p.chain || p.sh.is64) {
        for (size_t q = 0; q < steps.size(); ++q) FO_TRY(run_product(ctx, p, steps[q], s, tag, (int)q, run));
        return FO_OK;
    }
    const HostWork& w = p.wtc[p.tile_n == 128 ? 1 : 0];
    for (size_t q0 = 0; q0 < steps.size(); q0 += kMaxChain) {
        const int nq = (int)std::min<size_t>(kMaxChain, steps.size() - q0);
        const int h = prof_begin(ctx, s, FO_STAGE_PRODUCTS);
        int launches = 0;
        for (const Group& g : p.groups) {
            std::string err;
            cudaError_t e = tc_chain(p.key.prec, p.tile_n, p.tile_ctas, p.tile_drain, steps.data() + q0, nq, p.d_inst,
                                     p.d_io, w.dev.pre, w.pre.data(), g.i0, g.i1, p.maps.data() + 256 * (size_t)g.b0,
                                     g.b0, g.nb, ctx->flag, p.counters, p.chain_win, s, &err,
                                     p.key.sym ? (p.sh.ublk ? 2 : 1) : 0);
            if (e == cudaSuccess && debug_sync() && !ctx->capturing) e = cudaDeviceSynchronize();
            if (e != cudaSuccess) {
                const std::string where = std::string("tc_chain ") + tag;
                if (!err.empty()) return fail(ctx, FO_ERR_CUDA, where + ": " + err);
                return cuda_fail(ctx, e, where.c_str());
            }
            ++launches;
        }
        prof_end(ctx, s, h, p.flops_product * nq, launches);
        run->launches += launches;
        run->n_gemm += nq;
    }
    return FO_OK;
}

// The last Clenshaw or Horner step, which forms P. In the split forms its epilogue also leaves
// partials of tr P and ||P||_F^2 per 128 x 128 block. Without the trace correction it writes
// the caller's float64 P. With it, P goes to slot `pslot` instead (R_0's, read and then
// overwritten entry by entry, like every Clenshaw step's R_l -> b_l): the float32 master on
// both sides of the diagonal and the 16-bit planes, the operands of the correcting product
// P P, whose epilogue writes the caller's P from that master (the float64 P of this step is
// exactly the widening of its float32 values, so nothing is lost).
void final_step_extras(const Plan& p, Step& st, int pslot) {
    if (p.sh.is64) return;
    st.part = p.part_tc;
    st.part_pre = p.wtc[1].dev.pre;
    if (p.fix) {
        // P's float32 master on both sides of the diagonal, and the planes the correcting
        // product reads
        st.out = pslot;
        st.planes = fix_precision(p) == FO_PREC_BF16X1 ? 1 : p.sh.planes;
        st.lower_master = 1;
        st.out64 = 0;
    }
}

// Slot of T_{j k} for j >= 1: T_k is baby slot k-1, giants T_{2k}.. follow.
int giant_slot(const Plan& p, int j) { return j == 1 ? p.sh.k - 1 : p.sh.k + j - 2; }
int r_slot(const Plan& p, int l) { return p.sh.n_tslots + l; }

// The members U_1..U_jmax of a Chebyshev chain (U_j = T_j for the baby steps, U_j = T_{jk}
// for the giant steps; U_0 = I is a diagonal shift), given U_1, by
//  - the three-term recurrence U_{j+1} = 2 U_1 U_j - U_{j-1}, one product per launch
//    (sequential), or
//  - Algorithm 1 (staged): stage 1 computes U_2 = 2 U_1 U_1 - I; stage s >= 2, with
//    u = 2^{s-2}, v = 2^{s-1}, computes U_{i+u} = 2 U_i U_u - U_{i-u} and
//    U_{i+v} = 2 U_v U_i - U_{v-i} for u < i <= v, i.e. U_{v+1}..U_{2v} from U_1..U_v: the
//    products of a stage are independent and run as one launch.
// Either way jmax - 1 products; slot(j) gives the slot of U_j (j >= 1).
template <class SlotOf>
fo_status chebyshev_chain(fo_ctx* ctx, Plan& p, int jmax, SlotOf slot, bool staged, cudaStream_t s,
                          const char* tag, Run* run, bool giant = false) {
    auto prod = [&](int a, int b, int c, int out) {
        // 2 U_a U_b - U_c, U_0 = I
        return c == 0 ? make_step(p, slot(a), slot(b), -1, -1, slot(out), 2.0, 0.0, -1.0, false, false, false,
                                  false, ctx)
                      : make_step(p, slot(a), slot(b), slot(c), -1, slot(out), 2.0, -1.0, 0.0, false, false,
                                  false, false, ctx);
    };
    if (jmax < 2) return FO_OK;
    if (!staged) {
        std::vector<Step> chain;
        for (int j = 1; j < jmax; ++j) {
            chain.push_back(prod(1, j, j - 1, j + 1));
            // the giant step T_{(j+1)k} feeds the moments of expansions with m_eff > j + 1 only
            if (giant) chain.back().need_m = j + 1;
        }
        return run_chain(ctx, p, chain, s, tag, run);
    }
    {
        const Step st = prod(1, 1, 0, 2);
        FO_TRY(run_product(ctx, p, st, s, tag, 2, run));
    }
    for (int v = 2, u = 1; v < jmax; u = v, v *= 2) {
        std::vector<Step> stage;
        for (int i = u + 1; i <= v; ++i)
            if (i + u <= jmax) stage.push_back(prod(i, u, i - u, i + u));
        for (int i = u + 1; i <= v; ++i)
            if (i + v <= jmax) stage.push_back(prod(v, i, v - i, i + v));
        FO_TRY(run_products(ctx, p, stage.data(), (int)stage.size(), s, tag, 2 * v, run));
    }
    return FO_OK;
}

// Baby steps T_2..T_kmax.
fo_status baby_steps(fo_ctx* ctx, Plan& p, int kmax, cudaStream_t s, Run* run) {
    return chebyshev_chain(ctx, p, kmax, [](int j) { return j - 1; }, p.key.staged != 0, s, "baby", run);
}

// Giant steps T_{2k}..T_{(m-1)k}: the chain U_j = T_{jk} = T_j(T_k).
fo_status giant_steps(fo_ctx* ctx, Plan& p, cudaStream_t s, Run* run) {
    return chebyshev_chain(ctx, p, p.sh.m - 1, [&p](int j) { return giant_slot(p, j); }, p.key.staged != 0, s,
                           "giant", run, true);
}

// Exact moments tau_0..tau_{n_terms-1} (needs the giant steps).
fo_status exact_moments(fo_ctx* ctx, Plan& p, cudaStream_t s, Run* run) {
    const Shape& sh = p.sh;
    FO_CUDA(launch_diag_sums(p.d_inst, p.batch, sh.n_tslots, sh, s), "diag_sums");
    run->launches += 1;
    if (sh.m > 1 && sh.k > 1)
        FO_CUDA(launch_gram(p.d_inst, p.batch, p.wgr.dev, sh.k - 1, sh.m - 1, 0, sh.k - 1, 0, sh.is64,
                            sh.is64 ? nullptr : &p.gram_geom, ctx->flag, s,
                            &run->launches),
                "gram");
    FO_CUDA(launch_assemble_moments(p.d_inst, p.batch, sh, s), "moments");
    run->launches += 1;
    return FO_OK;
}

// Clenshaw recurrence in Y = T_k: b_{m-1} = R_{m-1}; b_l = 2 Y b_{l+1} - b_{l+2} + R_l;
// P = Y b_1 - b_2 + R_0 (written as float64 into the instance's P). b_l overwrites R_l.
fo_status clenshaw(fo_ctx* ctx, Plan& p, cudaStream_t s, Run* run) {
    const int m = p.sh.m;
    if (m == 1) return FO_OK;
    const int y = giant_slot(p, 1);
    std::vector<Step> chain;
    for (int l = m - 2; l >= 1; --l) {
        const bool has_c = l + 2 <= m - 1;
        chain.push_back(make_step(p, y, r_slot(p, l + 1), has_c ? r_slot(p, l + 2) : -1, r_slot(p, l), r_slot(p, l),
                                  2.0, has_c ? -1.0 : 0.0, 0.0, false, true, true, false, ctx));
        // an expansion cut at m_eff giant steps has b_l = R_l = 0 for l >= m_eff and
        // b_{m_eff - 1} = R_{m_eff - 1} (already in its slot): only l < m_eff - 1 is computed
        chain.back().need_m = l + 1;
    }
    const bool has_c = m >= 3;
    Step st = make_step(p, y, r_slot(p, 1), has_c ? r_slot(p, 2) : -1, r_slot(p, 0), -1, 1.0,
                        has_c ? -1.0 : 0.0, 0.0, false, true, false, true, ctx);
    final_step_extras(p, st, r_slot(p, 0));
    chain.push_back(st);
    return run_chain(ctx, p, chain, s, "clenshaw", run);
}

// Spectral bounds, X and the baby steps T_2..T_k of every instance.
fo_status front(fo_ctx* ctx, Plan& p, cudaStream_t s, Run* run) {
    const int h = prof_begin(ctx, s, FO_STAGE_BOUNDS);
    FO_CUDA(launch_bounds(p.d_inst, p.d_io, p.batch, p.wg.dev, p.part_g, p.key.use_given, s), "bounds");
    int l = (p.key.use_given ? 1 : 2) + 1;
    if (p.key.lanczos > 0 && !p.key.use_given)
        FO_CUDA(launch_lanczos(p.d_inst, p.d_io, p.batch, p.wg.dev, p.part_g, p.key.lanczos, s, &l), "lanczos");
    FO_CUDA(launch_scale(p.d_inst, p.d_io, p.wsc.dev, p.sh, s, ctx->flag + 1), "scale");
    prof_end(ctx, s, h, 0.0, l);
    run->launches += l;
    return baby_steps(ctx, p, p.sh.k, s, run);
}

// mu of every active instance from exact moments: giant steps, moments, DOS weights and the
// bracketed search (starting from the learned proposal when start_mu0 is set).
fo_status exact_mu(fo_ctx* ctx, Plan& p, cudaStream_t s, Run* run, int start_mu0) {
    if (p.giants) FO_TRY(giant_steps(ctx, p, s, run));
    int h = prof_begin(ctx, s, FO_STAGE_MOMENTS);
    const int l0 = run->launches;
    FO_TRY(exact_moments(ctx, p, s, run));
    prof_end(ctx, s, h, 0.0, run->launches - l0);
    h = prof_begin(ctx, s, FO_STAGE_MU);
    const int max_it = p.key.max_bisect > 0 ? p.key.max_bisect : 200;
    FO_CUDA(launch_dos_weights(p.d_inst, p.batch, p.sh, p.ct, s), "dos_weights");
    FO_CUDA(launch_bisect(p.d_inst, p.d_io, p.batch, p.sh, p.ct, max_it, start_mu0, s), "bisect");
    prof_end(ctx, s, h, 0.0, 2);
    run->launches += 2;
    return FO_OK;
}

// The paper's nested Horner form in the power basis of Y = T_k: Y_{m-1} = S_{m-1},
// Y_j = S_j + T_k Y_{j+1}, P = Y_0 (float64 into the instance's P); Y_j overwrites S_j.
fo_status horner(fo_ctx* ctx, Plan& p, cudaStream_t s, Run* run) {
    const int m = p.sh.m;
    if (m == 1) return FO_OK;
    const int y = giant_slot(p, 1);
    for (int j = m - 2; j >= 1; --j) {
        const Step st = make_step(p, y, r_slot(p, j + 1), -1, r_slot(p, j), r_slot(p, j), 1.0, 0.0, 0.0, false,
                                  true, true, false, ctx);
        FO_TRY(run_product(ctx, p, st, s, "horner", j, run));
    }
    Step st = make_step(p, y, r_slot(p, 1), -1, r_slot(p, 0), -1, 1.0, 0.0, 0.0, false, true, false, true, ctx);
    final_step_extras(p, st, r_slot(p, 0));
    return run_product(ctx, p, st, s, "horner", 0, run);
}

// tr P and ||P||_F^2 of every active instance after the float64-output product: from the
// product's partials per 128 x 128 block (split forms, m > 1), else by a pass over P. tmode 1
// also computes the trace correction's gamma (see trace_fix).
fo_status trace_stage(fo_ctx* ctx, Plan& p, cudaStream_t s, Run* run, int tmode) {
    const int h = prof_begin(ctx, s, FO_STAGE_TRACE);
    if (!p.sh.is64 && p.sh.m > 1) {
        FO_CUDA(launch_tile_trace(p.d_inst, p.d_io, p.batch, p.wtc[1].dev.pre, p.part_tc, tmode, s), "trace");
        prof_end(ctx, s, h, 0.0, 1);
        run->launches += 1;
    } else {
        FO_CUDA(launch_trace_frob(p.d_inst, p.d_io, p.wr.dev, p.part_t, s), "trace");
        prof_end(ctx, s, h, 0.0, 2);
        run->launches += 2;
    }
    return FO_OK;
}

// Trace correction of the split forms (after trace_stage with tmode 1 set gamma): the product
// P P whose epilogue writes the caller's float64 P = P + gamma (P - P P) (the first-order shift
// of mu that restores tr P = N_e; the small term in float32, added in float64), then the
// per-instance sum of the new trace and the removal of the product's own float64 residual by
// the trace projection (k_tile_trace, mode 2).
fo_status trace_fix(fo_ctx* ctx, Plan& p, cudaStream_t s, Run* run) {
    const int pslot = r_slot(p, 0);
    // A = B = P (planes), C = P's float32 master (beta 0: read by the correcting epilogue)
    Step st = make_step(p, pslot, pslot, pslot, -1, -1, 1.0, 0.0, 0.0, false, false, false, true, ctx);
    st.fix64 = 1;
    st.part = p.part_tc;
    st.part_pre = p.wtc[1].dev.pre;
    FO_TRY(run_product(ctx, p, st, s, "trace fix", 0, run, fix_precision(p)));
    return trace_stage(ctx, p, s, run, 2);
}

// P of every active instance at its current mu: coefficients, R_l, Clenshaw, tr P, ||P||^2
// (or, with the power basis, d_{i,j}, S_j and Horner). tmode as in trace_stage.
fo_status evaluate(fo_ctx* ctx, Plan& p, cudaStream_t s, Run* run, int poly_trace, int tmode) {
    const Shape& sh = p.sh;
    int h = prof_begin(ctx, s, FO_STAGE_COEFFS);
    int lstage = 0;
    FO_CUDA(launch_coefficients(p.d_inst, p.d_io, p.batch, sh, p.ct, poly_trace, s, &lstage), "coeffs");
    if (p.key.power) {
        FO_CUDA(launch_g_to_d(p.d_inst, p.batch, sh, s), "power-basis coefficients");
        lstage += 1;
    }
    prof_end(ctx, s, h, 0.0, lstage);
    run->launches += lstage;
    h = prof_begin(ctx, s, FO_STAGE_CONTRACT);
    lstage = sh.is64 ? 1 : (sh.m + 31) / 32 + (sh.m > 1 ? 1 : 0);   // + the plane mirror of R_{m-1}
    FO_CUDA(launch_contract(p.d_inst, p.we.dev, p.wct.dev, p.wsc.dev, sh, s, ctx->flag + 1), "contract");
    if (sh.m == 1) {
        FO_CUDA(launch_copy_out(p.d_inst, p.d_io, p.we.dev, sh, s), "copy_out");
        lstage += 1;
    }
    prof_end(ctx, s, h, 0.0, lstage);
    run->launches += lstage;
    FO_TRY(p.key.power ? horner(ctx, p, s, run) : clenshaw(ctx, p, s, run));
    return trace_stage(ctx, p, s, run, tmode);
}

// Learned mu: moments up to 2k from the baby steps, the network's proposal, evaluation of P
// and the trace judge; corrected re-evaluations; exact moments and bisection for whatever
// is still rejected. Eager calls stop as soon as every instance is accepted; a captured
// graph runs every round (rejected-free instances skip the work of each kernel).
// Moments up to 2k from the baby steps, the network's features, forward pass and proposal
// (mu, and with use_order the per-instance expansion order).
fo_status propose(fo_ctx* ctx, Plan& p, cudaStream_t s, Run* run, int use_order) {
    const Shape& sh = p.sh;
    const int B = p.batch;
    const MlpOffsets mo = mlp_offsets();
    const float* params = ctx->mlp;
    const float* norm = ctx->mlp + 4 * (size_t)mo.total;
    float* feat = p.lscratch;
    float* xn = feat + (size_t)B * kMlpIn;
    float* z1 = xn + (size_t)B * kMlpIn;
    float* a1 = z1 + (size_t)B * kMlpHidden;
    float* z2 = a1 + (size_t)B * kMlpHidden;
    float* a2 = z2 + (size_t)B * kMlpHidden;
    float* y = a2 + (size_t)B * kMlpHidden;
    int h = prof_begin(ctx, s, FO_STAGE_MOMENTS);
    int l0 = run->launches;
    FO_CUDA(launch_diag_sums(p.d_inst, B, sh.k, sh, s), "diag_sums");
    FO_CUDA(launch_gram(p.d_inst, B, p.wgr.dev, sh.k - 1, 1, 0, sh.k, 0, sh.is64,
                        sh.is64 ? nullptr : &p.gram_geom, ctx->flag, s, &run->launches), "gram");
    FO_CUDA(launch_assemble_low(p.d_inst, B, sh.k, s), "low moments");
    run->launches += 2;
    prof_end(ctx, s, h, 0.0, run->launches - l0);
    h = prof_begin(ctx, s, FO_STAGE_MU);
    FO_CUDA(launch_features(p.d_inst, p.d_io, B, sh.k, 0, feat, s), "features");
    FO_CUDA(mlp_gather_norm(feat, nullptr, B, kMlpIn, norm, norm + kMlpIn, xn, s), "normalise");
    FO_CUDA(mlp_forward(params, xn, B, z1, a1, z2, a2, y, s), "network");
    FO_CUDA(launch_learned_mu(p.d_inst, B, y, norm, sh.n_terms, sh.k, sh.m, use_order, kOrderMargin, s),
            "proposal");
    prof_end(ctx, s, h, 0.0, 6);
    run->launches += 6;
    return FO_OK;
}

fo_status learned(fo_ctx* ctx, Plan& p, cudaStream_t s, Run* run) {
    const Shape& sh = p.sh;
    const int B = p.batch;
    FO_TRY(propose(ctx, p, s, run, 0));
    const int R = p.key.max_newton == 0 ? 2 : (p.key.max_newton < 0 ? 0 : p.key.max_newton);
    bool any = true;
    for (int r = 0; r <= R; ++r) {
        FO_TRY(evaluate(ctx, p, s, run, 0, 0));
        if (r < R) {
            FO_CUDA(launch_poly_width(p.d_inst, B, sh, p.ct, s), "expansion width");
            run->launches += 1;
        }
        FO_CUDA(cudaMemsetAsync(p.lcount, 0, sizeof(int), s), "judge");
        FO_CUDA(launch_learned_check(p.d_inst, p.d_io, B, r, R, p.key.tr_tol, sh.is64, p.lcount, s), "judge");
        run->launches += 1;
        if (!ctx->capturing) {
            FO_CUDA(cudaMemcpyAsync(ctx->hcount, p.lcount, sizeof(int), cudaMemcpyDeviceToHost, s), "judge");
            FO_CUDA(cudaStreamSynchronize(s), "judge");
            any = *ctx->hcount > 0;
            if (!any) break;
        }
    }
    if (any) {
        FO_TRY(exact_mu(ctx, p, s, run, 1));
        FO_TRY(evaluate(ctx, p, s, run, 1, 0));
    }
    if (p.fix) {
        // every instance's partials are those of its last evaluation (accepted instances are
        // skipped by later ones): gamma for all of them, then the correcting product
        FO_TRY(trace_stage(ctx, p, s, run, 1));
        FO_TRY(trace_fix(ctx, p, s, run));
    }
    return FO_OK;
}

// Learned expansion order: the network proposes each instance's order, the expansion is cut
// there (coefficients from n_eff on are zero, the giant and Clenshaw products it leaves zero
// or unused are skipped), and mu is the bisection's on the exact moments of that expansion,
// started from the network's mu; the trace correction follows as for bisection.
fo_status learned_order(fo_ctx* ctx, Plan& p, cudaStream_t s, Run* run) {
    FO_TRY(propose(ctx, p, s, run, 1));
    FO_TRY(exact_mu(ctx, p, s, run, 1));
    FO_TRY(evaluate(ctx, p, s, run, 1, p.fix ? 1 : 0));
    return p.fix ? trace_fix(ctx, p, s, run) : FO_OK;
}

// The whole method for every instance of a density plan (after the per-call inputs).
fo_status run_density(fo_ctx* ctx, Plan& p, cudaStream_t s, Run* run) {
    FO_TRY(front(ctx, p, s, run));
    switch (p.key.mu_mode) {
        case FO_MU_BISECT:
            FO_TRY(exact_mu(ctx, p, s, run, 0));
            FO_TRY(evaluate(ctx, p, s, run, 1, p.fix ? 1 : 0));
            return p.fix ? trace_fix(ctx, p, s, run) : FO_OK;
        case FO_MU_LEARNED:
            return learned(ctx, p, s, run);
        case FO_MU_ORDER:
            return learned_order(ctx, p, s, run);
        default:
            FO_CUDA(launch_set_mu(p.d_inst, p.d_io, p.batch, s), "mu");
            run->launches += 1;
            return evaluate(ctx, p, s, run, 0, 0);
    }
}

// Tile configuration of the tensor-core products: the requested one, or the fastest of
// (256 wide, 1 CTA/SM, 8 or 16 drain warps), (128 wide, 1 CTA/SM) and (128 wide, 2 CTAs/SM)
// on this plan's first baby step, timed with CUDA events on the plan's own layout (the data
// are whatever the workspace holds; the work does not depend on them).
fo_status autotune(fo_ctx* ctx, Plan& p) {
    constexpr int kTuneReps = 5;   // timed products per candidate (the storages differ by a few per cent)
    p.sh.ublk = 0;
    if (p.sh.is64 || p.n_slots == 0) {
        p.tile_n = p.tile_ctas = p.tile_drain = p.tile_store = 0;
        return FO_OK;
    }
    if (p.key.tile_req) {
        p.tile_n = p.key.tile_req;
        p.tile_ctas = p.key.ctas_req ? p.key.ctas_req : 1;
        p.tile_drain = p.key.drain_req ? p.key.drain_req : 8;
        p.tile_store = (p.key.store_req == 2 && p.key.sym) ? 2 : 1;
        p.tile_persist = p.key.persist_req == 2 ? 1 : 0;
        p.sh.ublk = p.tile_store == 2;
        return FO_OK;
    }
    if (p.key.mode == MODE_PRODUCT || p.sh.k < 2) {
        p.tile_n = 256;
        p.tile_ctas = 1;
        p.tile_drain = 8;
        p.tile_store = 1;
        return FO_OK;
    }
    // make every instance active (the per-call inputs are not needed by a product)
    std::vector<InstIO> io(p.batch);
    std::memset(io.data(), 0, sizeof(InstIO) * io.size());
    cudaStream_t s = nullptr;
    FO_CUDA(launch_set_io(io.data(), p.batch, p.d_io, p.d_inst, 0, s), "autotune setup");
    const Step st = make_step(p, 0, 0, -1, -1, 1, 2.0, 0.0, -1.0, false, false, false, false, ctx);
    cudaEvent_t e0 = ev_get(ctx), e1 = ev_get(ctx);
    float best = 0.0f;
    int bn = 256, bc = 1, bd = 8, bs = 1;
    const bool prof = ctx->prof;
    ctx->prof = false;
    // tile width, CTAs per SM, drain warps, plane storage (the upper-block storage trades the
    // mirrored epilogue writes for transposed operand loads: it pays on short tiles), and the
    // persistent kernel (128-wide tiles; its epilogue overlaps the next tile's products)
    const int cands[12][5] = {{256, 1, 8, 1, 0}, {256, 1, 16, 1, 0}, {128, 1, 8, 1, 0}, {128, 2, 8, 1, 0},
                              {128, 1, 8, 1, 1}, {256, 1, 8, 2, 0}, {256, 1, 16, 2, 0}, {128, 1, 8, 2, 0},
                              {128, 2, 8, 2, 0}, {128, 1, 8, 2, 1}};
    const int ncand = p.key.sym ? 10 : 5;
    int bp = 0;
    for (int ci = 0; ci < ncand; ++ci) {
        // the persistent kernel is timed only when asked for: measured slower on every workload
        // here (its one CTA per SM cannot feed 128-wide split-precision tiles as two
        // co-resident CTAs do)
        if (p.key.persist_req != 2 && cands[ci][4]) continue;
        if (p.key.persist_req == 2 && !cands[ci][4]) continue;
        p.tile_n = cands[ci][0];
        p.tile_ctas = cands[ci][1];
        p.tile_drain = cands[ci][2];
        p.tile_persist = cands[ci][4];
        p.sh.ublk = cands[ci][3] == 2;
        Run r;
        fo_status rs = run_product(ctx, p, st, s, "autotune", ci, &r);   // warm-up
        if (rs != FO_OK) { ctx->prof = prof; return rs; }
        cudaEventRecord(e0, s);
        for (int rep = 0; rep < kTuneReps; ++rep) {
            rs = run_product(ctx, p, st, s, "autotune", ci, &r);
            if (rs != FO_OK) { ctx->prof = prof; return rs; }
        }
        cudaEventRecord(e1, s);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            ctx->prof = prof;
            return fail(ctx, FO_ERR_CUDA, "autotune timing failed");
        }
        if (autotune_log())
            std::fprintf(stderr, "autotune n0=%lld batch=%d tile %dx%dx%d store %d persistent %d: %.4f ms per product\n",
                         (long long)p.key.n[0], p.batch, cands[ci][0], cands[ci][1], cands[ci][2], cands[ci][3],
                         cands[ci][4], ms / kTuneReps);
        if (best == 0.0f || ms < best) {
            best = ms;
            bn = cands[ci][0];
            bc = cands[ci][1];
            bd = cands[ci][2];
            bs = cands[ci][3];
            bp = cands[ci][4];
        }
    }
    ctx->prof = prof;
    ctx->ev_pool.push_back(e0);
    ctx->ev_pool.push_back(e1);
    int flag = 0;
    FO_CUDA(cudaMemcpy(&flag, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost), "autotune flag");
    if (flag) return fail(ctx, FO_ERR_DEVICE_TIMEOUT, "tensor-core wait timed out during autotuning");
    p.tile_n = bn;
    p.tile_ctas = bc;
    p.tile_drain = bd;
    p.tile_store = bs;
    p.tile_persist = bp;
    p.sh.ublk = bs == 2;
    return FO_OK;
}

fo_status get_plan(fo_ctx* ctx, const PlanKey& key, Plan** out) {
    for (size_t i = 0; i < ctx->plans.size(); ++i) {
        if (ctx->plans[i]->key == key && ctx->plans[i]->ws_gen == ctx->ws_gen) {
            std::unique_ptr<Plan> p = std::move(ctx->plans[i]);
            ctx->plans.erase(ctx->plans.begin() + i);
            ctx->plans.push_back(std::move(p));
            *out = ctx->plans.back().get();
            return FO_OK;
        }
    }
    std::unique_ptr<Plan> p(new (std::nothrow) Plan());
    if (!p) return fail(ctx, FO_ERR_NOMEM, "plan allocation failed");
    FO_TRY(layout_plan(ctx, key, p.get()));
    FO_TRY(ensure_ws(ctx, p->total));
    // stale plans (older workspace) and the least recently used beyond the cap
    bool stale = false;
    for (auto& q : ctx->plans) stale |= q->ws_gen != ctx->ws_gen;
    if (stale || ctx->plans.size() >= kMaxPlans) cudaDeviceSynchronize();
    ctx->plans.erase(std::remove_if(ctx->plans.begin(), ctx->plans.end(),
                                    [&](const std::unique_ptr<Plan>& q) { return q->ws_gen != ctx->ws_gen; }),
                     ctx->plans.end());
    while (ctx->plans.size() >= kMaxPlans) ctx->plans.erase(ctx->plans.begin());
    FO_TRY(place_plan(ctx, p.get()));
    FO_TRY(autotune(ctx, *p));
    ctx->plans.push_back(std::move(p));
    *out = ctx->plans.back().get();
    return FO_OK;
}

fo_status check_params(fo_ctx* ctx, const fo_params* prm) {
    if (!prm) return fail(ctx, FO_ERR_ARG, "params is NULL");
    if (!(prm->kT > 0.0) || !std::isfinite(prm->kT)) return fail(ctx, FO_ERR_ARG, "kT must be > 0");
    if (prm->use_given_bounds && !(prm->emax > prm->emin))
        return fail(ctx, FO_ERR_ARG, "emax must exceed emin");
    if (prm->mu_mode < FO_MU_FIXED || prm->mu_mode > FO_MU_ORDER)
        return fail(ctx, FO_ERR_ARG, "unknown mu_mode");
    if ((prm->mu_mode == FO_MU_LEARNED || prm->mu_mode == FO_MU_ORDER) && !ctx->mlp_ready)
        return fail(ctx, FO_ERR_UNSUPPORTED, "learned mu needs a trained, loaded or set model");
    if (prm->mu_mode == FO_MU_LEARNED && !(prm->tr_tol >= 0.0)) return fail(ctx, FO_ERR_ARG, "tr_tol must be >= 0");
    if (prm->tile_n != 0 && prm->tile_n != 128 && prm->tile_n != 256)
        return fail(ctx, FO_ERR_ARG, "tile_n must be 0, 128 or 256");
    if (prm->tile_drain != 0 && (prm->tile_drain != 8 && prm->tile_drain != 16))
        return fail(ctx, FO_ERR_ARG, "tile_drain must be 0, 8 or 16");
    if (prm->tile_drain == 16 && prm->tile_n != 256)
        return fail(ctx, FO_ERR_ARG, "16 drain warps need tile_n = 256");
    if ((prm->flags & FO_FLAG_POWER_BASIS) && prm->precision == FO_PREC_FP16X2)
        return fail(ctx, FO_ERR_UNSUPPORTED, "the power basis overflows the fp16 range");
    if (prm->precision != FO_PREC_FP64 && !(prm->flags & FO_FLAG_ALLOW_LOOSE)) {
        // combinations measured beyond the split forms' 1e-6 bar run only on request
        if (prm->flags & FO_FLAG_STAGED)
            return fail(ctx, FO_ERR_UNSUPPORTED,
                        "staged chains in a split precision exceed the 1e-6 bar (set FO_FLAG_ALLOW_LOOSE)");
        if (prm->flags & FO_FLAG_POWER_BASIS)
            return fail(ctx, FO_ERR_UNSUPPORTED,
                        "the power basis in a split precision exceeds the 1e-6 bar (set FO_FLAG_ALLOW_LOOSE)");
        int k = 0, m = 0;
        if (prm->k > 0 && plan_km(prm->n_terms, prm->k, &k, &m) && m > k)
            return fail(ctx, FO_ERR_UNSUPPORTED,
                        "k below ceil(sqrt(n_terms)) lengthens the Clenshaw chain beyond the split forms' "
                        "1e-6 bar (set FO_FLAG_ALLOW_LOOSE)");
    }
    if (prm->lanczos_steps < 0 || prm->lanczos_steps > kLzMax)
        return fail(ctx, FO_ERR_ARG, "lanczos_steps must be in [0, 64]");
    if (prm->tile_ctas < 0 || prm->tile_ctas > 2 || (prm->tile_ctas == 2 && prm->tile_n != 128) ||
        (prm->tile_ctas != 0 && prm->tile_n == 0))
        return fail(ctx, FO_ERR_ARG, "tile_ctas must be 0, 1 or 2 (2 with tile_n = 128), set with tile_n");
    if (prm->tile_store < 0 || prm->tile_store > 2 || (prm->tile_store != 0 && prm->tile_n == 0))
        return fail(ctx, FO_ERR_ARG, "tile_store must be 0, 1 or 2, set with tile_n");
    if (prm->chain < 0 || prm->chain > 2 || prm->chain_window < 0)
        return fail(ctx, FO_ERR_ARG, "chain must be 0, 1 or 2 and chain_window >= 0");
    if (prm->tile_persist < 0 || prm->tile_persist > 2 ||
        (prm->tile_persist == 2 && prm->tile_n != 0 && (prm->tile_n != 128 || prm->tile_ctas == 2)))
        return fail(ctx, FO_ERR_ARG, "tile_persist must be 0, 1 or 2 (2 with 128-wide tiles, 1 CTA per SM)");
    return FO_OK;
}

fo_status ensure_hres(fo_ctx* ctx, size_t count) {
    if (ctx->hres_count >= count) return FO_OK;
    if (ctx->hres) cudaFreeHost(ctx->hres);
    ctx->hres = nullptr;
    ctx->hres_count = 0;
    if (cudaMallocHost(&ctx->hres, sizeof(DevResult) * count) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, FO_ERR_NOMEM, "pinned readback buffer allocation failed");
    }
    ctx->hres_count = count;
    return FO_OK;
}

// Density matrices of `batch` instances (caller order) on one plan.
fo_status density_batch(fo_ctx* ctx, int batch, const double* const* dH, const int64_t* n, const int64_t* ld,
                        const double* n_e, const double* kT, const fo_params* prm, double* const* dP,
                        const int64_t* ldp, fo_result* res, cudaStream_t st) {
    FO_TRY(check_params(ctx, prm));
    if (batch < 1 || !dH || !dP || !n || !n_e) return fail(ctx, FO_ERR_ARG, "bad batch arguments");
    const bool bisect = prm->mu_mode != FO_MU_FIXED;
    for (int b = 0; b < batch; ++b) {
        if (!dH[b] || !dP[b]) return fail(ctx, FO_ERR_ARG, "H and P must be non-NULL");
        if (n[b] < 1) return fail(ctx, FO_ERR_ARG, "n must be >= 1");
        if ((ld && ld[b] < n[b]) || (ldp && ldp[b] < n[b]))
            return fail(ctx, FO_ERR_ARG, "leading dimensions must be >= n");
        if (bisect && !(n_e[b] >= 0.0 && n_e[b] <= (double)n[b]))
            return fail(ctx, FO_ERR_ARG, "n_e must be in [0, n]");
        if (kT && (!(kT[b] > 0.0) || !std::isfinite(kT[b]))) return fail(ctx, FO_ERR_ARG, "kT must be > 0");
    }
    // a device timeout of an earlier call is reported by that call: clear it for this one
    FO_CUDA(cudaMemsetAsync(ctx->flag, 0, sizeof(int), st), "reset the timeout flag");
    PlanKey key;
    key.n.assign(n, n + batch);
    key.mode = MODE_DENSITY;
    key.n_terms = prm->n_terms;
    key.k_req = prm->k;
    key.prec = prm->precision;
    key.mu_mode = prm->mu_mode;
    key.n_quad = prm->n_quad;
    key.use_given = prm->use_given_bounds ? 1 : 0;
    key.tile_req = prm->tile_n;
    key.ctas_req = prm->tile_ctas;
    key.drain_req = prm->tile_drain;
    key.store_req = prm->tile_store;
    key.max_bisect = prm->max_bisect;
    key.staged = (prm->flags & FO_FLAG_STAGED) ? 1 : 0;
    key.lanczos = prm->lanczos_steps;
    key.power = (prm->flags & FO_FLAG_POWER_BASIS) ? 1 : 0;
    key.nofix = (prm->flags & FO_FLAG_NO_TRACE_FIX) ? 1 : 0;
    key.chain = prm->chain;
    key.chain_win = prm->chain_window;
    key.persist_req = prm->tile_persist;
    if (prm->mu_mode == FO_MU_LEARNED) {
        key.max_newton = prm->max_newton;
        key.tr_tol = prm->tr_tol;
    }
    Plan* p = nullptr;
    FO_TRY(get_plan(ctx, key, &p));

    std::vector<InstIO> io(batch);
    for (int j = 0; j < batch; ++j) {
        const int b = p->order[j];
        InstIO& x = io[j];
        std::memset(&x, 0, sizeof(x));
        x.H = dH[b];
        x.P = dP[b];
        x.ldh = ld ? ld[b] : n[b];
        x.ldp = ldp ? ldp[b] : n[b];
        x.kT = kT ? kT[b] : prm->kT;
        x.n_e = n_e[b];
        x.mu = prm->mu;
        x.emin = prm->emin;
        x.emax = prm->emax;
    }
    Run run;
    const int hcall = prof_begin(ctx, st, FO_STAGE_CALL);
    FO_CUDA(launch_set_io(io.data(), batch, p->d_io, p->d_inst, 0, st), "set_io");
    run.launches += (batch + 63) / 64;
    const bool graph = (prm->flags & FO_FLAG_GRAPH) != 0;
    if (graph) {
        if (!p->graph) {
            if (!ctx->cap) FO_CUDA(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking), "capture stream");
            FO_CUDA(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
            ctx->capturing = true;
            Run cap_run;
            const fo_status rs = run_density(ctx, *p, ctx->cap, &cap_run);
            cudaGraph_t g = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(ctx->cap, &g);
            ctx->capturing = false;
            if (rs != FO_OK) {
                if (g) cudaGraphDestroy(g);
                return rs;
            }
            if (ce != cudaSuccess) return cuda_fail(ctx, ce, "end capture");
            p->graph_launches = cap_run.launches;
            const cudaError_t ie = cudaGraphInstantiate(&p->graph, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                p->graph = nullptr;
                return cuda_fail(ctx, ie, "graph instantiate");
            }
        }
        FO_CUDA(cudaGraphLaunch(p->graph, st), "graph launch");
        // the graph holds the same launches as an eager call
        run.n_gemm = (p->sh.k - 1) + (p->giants ? p->sh.m - 2 : 0) + (p->sh.m > 1 ? p->sh.m - 1 : 0) +
                     (p->fix ? 1 : 0);
        run.launches += p->graph_launches;
    } else {
        FO_TRY(run_density(ctx, *p, st, &run));
    }
    prof_end(ctx, st, hcall, p->flops_product * run.n_gemm, run.launches);
    if (ctx->prof) ctx->prof_calls += 1;

    if (res && !(prm->flags & FO_FLAG_NO_RESULT_SYNC)) {
        FO_TRY(ensure_hres(ctx, batch));
        int flag[4] = {0, 0, 0, 0};
        FO_CUDA(cudaMemcpyAsync(ctx->hres, p->d_res, sizeof(DevResult) * batch, cudaMemcpyDeviceToHost, st),
                "readback");
        FO_CUDA(cudaMemcpyAsync(flag, ctx->flag, sizeof(flag), cudaMemcpyDeviceToHost, st), "readback");
        FO_CUDA(cudaStreamSynchronize(st), "sync");
        if (flag[1] != 0)
            return fail(ctx, FO_ERR_CUDA, "self-check violation code " + std::to_string(flag[1]) + " (" +
                                              std::to_string(flag[2]) + ", " + std::to_string(flag[3]) + ")");
        fo_status first = FO_OK;
        for (int j = 0; j < batch; ++j) {
            const DevResult& hr = ctx->hres[j];
            fo_result& r = res[p->order[j]];
            std::memset(&r, 0, sizeof(r));
            r.mu = hr.mu;
            r.trace = hr.trace;
            r.trace_raw = hr.trace_raw;
            r.trace_gamma = hr.gamma;
            r.trace_proj = hr.proj;
            r.trace_poly = hr.trace_poly;
            r.frob2 = hr.frob2;
            r.emin = hr.bounds[0];
            r.emax = hr.bounds[1];
            r.k = p->sh.k;
            r.m = p->sh.m;
            r.n_gemm = run.n_gemm;
            r.bisect_iters = hr.iters;
            r.learned_accepted = hr.learned_ok;
            r.n_launches = run.launches;
            r.tile_n = p->tile_n;
            r.tile_ctas = p->tile_ctas;
            r.tile_drain = p->tile_drain;
            r.tile_store = p->tile_store;
            r.tile_persist = p->tile_persist ? 2 : (p->tile_n ? 1 : 0);
            r.evals = 1;
            r.order = 0;
            if (prm->mu_mode == FO_MU_LEARNED) {
                // products of this instance: baby steps, one Clenshaw pass per evaluation,
                // and the giant steps of the exact fallback
                const int ev = hr.evals + (hr.learned_ok ? 0 : 1);
                const int km1 = p->sh.m > 1 ? p->sh.m - 1 : 0;
                r.evals = ev;
                r.n_gemm = (p->sh.k - 1) + ev * km1 + (hr.learned_ok ? 0 : (p->giants ? p->sh.m - 2 : 0)) +
                           (p->fix ? 1 : 0);
                r.order = (int)std::lround(hr.order);
                if (!hr.learned_ok) r.bisect_iters = hr.iters;
                else r.bisect_iters = 0;
            }
            if (prm->mu_mode == FO_MU_ORDER) {
                // the instance's own expansion: k - 1 baby steps, m_eff - 2 giant steps,
                // m_eff - 1 Clenshaw steps (and the trace correction)
                const int me = hr.m_eff > 0 ? hr.m_eff : p->sh.m;
                r.n_gemm = (p->sh.k - 1) + (p->giants ? std::max(0, me - 2) : 0) + (me > 1 ? me - 1 : 0) +
                           (p->fix ? 1 : 0);
                r.order = hr.n_eff > 0 ? hr.n_eff : p->sh.n_terms;
                r.m = me;
            }
            int status = hr.status;
            if (flag[0]) status = FO_ERR_DEVICE_TIMEOUT;
            r.status = status;
            if (status != FO_OK && first == FO_OK) first = (fo_status)status;
        }
        if (first != FO_OK)
            return fail(ctx, first, std::string("device stage failed: ") + fo_status_string(first));
    }
    return FO_OK;
}

// ---------------------------------------------------------------- learned model
size_t mlp_floats() { return 4 * (size_t)mlp_offsets().total + kMlpNorm; }
float* mlp_params(fo_ctx* ctx) { return ctx->mlp; }
float* mlp_grad(fo_ctx* ctx) { return ctx->mlp + mlp_offsets().total; }
float* mlp_m(fo_ctx* ctx) { return ctx->mlp + 2 * (size_t)mlp_offsets().total; }
float* mlp_v(fo_ctx* ctx) { return ctx->mlp + 3 * (size_t)mlp_offsets().total; }
float* mlp_norm(fo_ctx* ctx) { return ctx->mlp + 4 * (size_t)mlp_offsets().total; }

fo_status ensure_mlp(fo_ctx* ctx) {
    if (ctx->mlp) return FO_OK;
    if (cudaMalloc(&ctx->mlp, sizeof(float) * mlp_floats()) != cudaSuccess) {
        cudaGetLastError();
        ctx->mlp = nullptr;
        return fail(ctx, FO_ERR_NOMEM, "model allocation failed");
    }
    if (cudaMemset(ctx->mlp, 0, sizeof(float) * mlp_floats()) != cudaSuccess)
        return fail(ctx, FO_ERR_CUDA, "model clear failed");
    return FO_OK;
}

fo_status ensure_mlp_scratch(fo_ctx* ctx, size_t floats) {
    if (ctx->mlp_scratch_floats >= floats) return FO_OK;
    if (ctx->mlp_scratch) {
        cudaDeviceSynchronize();
        cudaFree(ctx->mlp_scratch);
    }
    ctx->mlp_scratch = nullptr;
    ctx->mlp_scratch_floats = 0;
    if (cudaMalloc(&ctx->mlp_scratch, sizeof(float) * floats) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, FO_ERR_NOMEM, "model scratch allocation failed");
    }
    ctx->mlp_scratch_floats = floats;
    return FO_OK;
}

// splitmix64 (Steele, Lea and Flood 2014): the counter-based generator of the weight
// initialisation and of the mini-batch order.
uint64_t splitmix64(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double unit_uniform(uint64_t& x) { return (double)(splitmix64(x) >> 11) * (1.0 / 9007199254740992.0); }

// Uniform(-a, a) weights, a = sqrt(6 / (fan_in + fan_out)); zero biases; identity normalisation.
void init_host_params(uint64_t seed, std::vector<float>& prm, std::vector<float>& norm) {
    const MlpOffsets o = mlp_offsets();
    prm.assign(o.total, 0.0f);
    uint64_t st = seed;
    auto fill = [&](int off, int fan_out, int fan_in) {
        const double a = std::sqrt(6.0 / (fan_in + fan_out));
        for (int q = 0; q < fan_out * fan_in; ++q) prm[off + q] = (float)((2.0 * unit_uniform(st) - 1.0) * a);
    };
    fill(o.W1, kMlpHidden, kMlpIn);
    fill(o.W2, kMlpHidden, kMlpHidden);
    fill(o.W3, kMlpOut, kMlpHidden);
    norm.assign(kMlpNorm, 0.0f);
    for (int c = 0; c < kMlpIn; ++c) norm[kMlpIn + c] = 1.0f;
    for (int c = 0; c < kMlpOut; ++c) norm[2 * kMlpIn + kMlpOut + c] = 1.0f;
}

fo_status upload_model(fo_ctx* ctx, const float* prm, const float* norm) {
    FO_TRY(ensure_mlp(ctx));
    const MlpOffsets o = mlp_offsets();
    if (cudaMemcpy(mlp_params(ctx), prm, sizeof(float) * o.total, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(mlp_norm(ctx), norm, sizeof(float) * kMlpNorm, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(mlp_m(ctx), 0, sizeof(float) * o.total) != cudaSuccess ||
        cudaMemset(mlp_v(ctx), 0, sizeof(float) * o.total) != cudaSuccess)
        return fail(ctx, FO_ERR_CUDA, "model upload failed");
    ctx->mlp_step = 0;
    ctx->mlp_ready = true;
    return FO_OK;
}

// Training pairs of a batch: the exact method (bisection on exact moments) gives mu; the
// features come from the same moments, the targets from mu, the coefficients at mu and the
// moments. P is not formed.
fo_status features_batch(fo_ctx* ctx, int batch, const double* const* dH, const int64_t* n, const int64_t* ld,
                         const double* n_e, const double* kT, const fo_params* prm, float* d_feat, float* d_tgt,
                         fo_result* res, cudaStream_t st) {
    fo_params q = *prm;
    q.mu_mode = FO_MU_BISECT;
    q.flags = 0;
    FO_TRY(check_params(ctx, &q));
    if (batch < 1 || !dH || !n || !n_e || !d_feat) return fail(ctx, FO_ERR_ARG, "bad batch arguments");
    for (int b = 0; b < batch; ++b) {
        if (!dH[b] || n[b] < 1 || (ld && ld[b] < n[b])) return fail(ctx, FO_ERR_ARG, "bad instance arguments");
        if (!(n_e[b] >= 0.0 && n_e[b] <= (double)n[b])) return fail(ctx, FO_ERR_ARG, "n_e must be in [0, n]");
        if (kT && (!(kT[b] > 0.0) || !std::isfinite(kT[b]))) return fail(ctx, FO_ERR_ARG, "kT must be > 0");
    }
    PlanKey key;
    key.n.assign(n, n + batch);
    key.mode = MODE_DENSITY;
    key.n_terms = q.n_terms;
    key.k_req = q.k;
    key.prec = q.precision;
    key.mu_mode = FO_MU_BISECT;
    key.n_quad = q.n_quad;
    key.use_given = q.use_given_bounds ? 1 : 0;
    key.tile_req = q.tile_n;
    key.ctas_req = q.tile_ctas;
    key.drain_req = q.tile_drain;
    key.store_req = q.tile_store;
    key.max_bisect = q.max_bisect;
    key.staged = (prm->flags & FO_FLAG_STAGED) ? 1 : 0;
    key.lanczos = q.lanczos_steps;
    Plan* p = nullptr;
    FO_TRY(get_plan(ctx, key, &p));
    std::vector<InstIO> io(batch);
    for (int j = 0; j < batch; ++j) {
        const int b = p->order[j];
        InstIO& x = io[j];
        std::memset(&x, 0, sizeof(x));
        x.H = dH[b];
        x.ldh = ld ? ld[b] : n[b];
        x.kT = kT ? kT[b] : q.kT;
        x.n_e = n_e[b];
        x.emin = q.emin;
        x.emax = q.emax;
    }
    Run run;
    FO_CUDA(launch_set_io(io.data(), batch, p->d_io, p->d_inst, 0, st), "set_io");
    FO_TRY(front(ctx, *p, st, &run));
    FO_TRY(exact_mu(ctx, *p, st, &run, 0));
    int l = 0;
    FO_CUDA(launch_coefficients(p->d_inst, p->d_io, batch, p->sh, p->ct, 1, st, &l), "coeffs");
    FO_CUDA(launch_features(p->d_inst, p->d_io, batch, p->sh.k, 1, d_feat, st), "features");
    if (d_tgt) FO_CUDA(launch_targets(p->d_inst, batch, p->sh.n_terms, d_tgt, st), "targets");
    if (res) {
        FO_TRY(ensure_hres(ctx, batch));
        FO_CUDA(cudaMemcpyAsync(ctx->hres, p->d_res, sizeof(DevResult) * batch, cudaMemcpyDeviceToHost, st),
                "readback");
        FO_CUDA(cudaStreamSynchronize(st), "sync");
        fo_status first = FO_OK;
        for (int j = 0; j < batch; ++j) {
            const DevResult& hr = ctx->hres[j];
            fo_result& r = res[p->order[j]];
            std::memset(&r, 0, sizeof(r));
            r.mu = hr.mu;
            r.trace_poly = hr.trace_poly;
            r.emin = hr.bounds[0];
            r.emax = hr.bounds[1];
            r.k = p->sh.k;
            r.m = p->sh.m;
            r.n_gemm = (p->sh.k - 1) + (p->giants ? p->sh.m - 2 : 0);
            r.bisect_iters = hr.iters;
            r.status = hr.status;
            r.tile_n = p->tile_n;
            r.tile_ctas = p->tile_ctas;
            if (hr.status != FO_OK && first == FO_OK) first = (fo_status)hr.status;
        }
        if (first != FO_OK) return fail(ctx, first, std::string("device stage failed: ") + fo_status_string(first));
    }
    return FO_OK;
}

}  // namespace

extern "C" {

const char* fo_version(void) { return "fermi-gb300 0.2"; }

const char* fo_status_string(fo_status s) {
    switch (s) {
        case FO_OK: return "ok";
        case FO_ERR_ARG: return "invalid argument";
        case FO_ERR_CUDA: return "CUDA error";
        case FO_ERR_NOMEM: return "out of device memory";
        case FO_ERR_NONFINITE: return "non-finite input";
        case FO_ERR_NO_BRACKET: return "mu not bracketed";
        case FO_ERR_NOT_CONVERGED: return "mu bisection not converged";
        case FO_ERR_DEVICE_TIMEOUT: return "device wait timed out";
        case FO_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* fo_last_error(const fo_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

fo_status fo_create(fo_ctx** out, int device) {
    if (!out) return FO_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return FO_ERR_CUDA;
    }
    fo_ctx* ctx = new (std::nothrow) fo_ctx();
    if (!ctx) return FO_ERR_NOMEM;
    ctx->device = device;
    DeviceGuard g(device);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&ctx->flag, 8 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return FO_ERR_NOMEM;
    }
    cudaMemset(ctx->flag, 0, 8 * sizeof(int));
    if (cudaMallocHost(&ctx->hcount, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ctx->flag);
        delete ctx;
        return FO_ERR_NOMEM;
    }
    *out = ctx;
    return FO_OK;
}

fo_status fo_destroy(fo_ctx* ctx) {
    if (!ctx) return FO_OK;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        prof_collect(ctx);
        ctx->plans.clear();
        for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
        if (ctx->ws) cudaFree(ctx->ws);
        for (auto& hs : ctx->hslot) {
            if (hs.buf) cudaFree(hs.buf);
            for (cudaEvent_t e : {hs.in, hs.done, hs.out})
                if (e) cudaEventDestroy(e);
        }
        if (ctx->h2d) cudaStreamDestroy(ctx->h2d);
        if (ctx->d2h) cudaStreamDestroy(ctx->d2h);
        if (ctx->flag) cudaFree(ctx->flag);
        if (ctx->hres) cudaFreeHost(ctx->hres);
        if (ctx->cap) cudaStreamDestroy(ctx->cap);
        if (ctx->hcount) cudaFreeHost(ctx->hcount);
        if (ctx->mlp) cudaFree(ctx->mlp);
        if (ctx->mlp_scratch) cudaFree(ctx->mlp_scratch);
    }
    delete ctx;
    return FO_OK;
}

fo_status fo_spectral_bounds(fo_ctx* ctx, const double* dH, int64_t n, int64_t ld, double* d_bounds,
                             void* stream) {
    if (!ctx) return FO_ERR_ARG;
    if (!dH || !d_bounds || n < 1 || ld < n) return fail(ctx, FO_ERR_ARG, "bad arguments");
    DeviceGuard g(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PlanKey key;
    key.n = {n};
    key.mode = MODE_BOUNDS;
    Plan* p = nullptr;
    FO_TRY(get_plan(ctx, key, &p));
    InstIO io;
    std::memset(&io, 0, sizeof(io));
    io.H = dH;
    io.ldh = ld;
    FO_CUDA(launch_set_io(&io, 1, p->d_io, p->d_inst, 0, st), "set_io");
    FO_CUDA(launch_bounds(p->d_inst, p->d_io, 1, p->wg.dev, p->part_g, 0, st), "bounds");
    FO_CUDA(launch_export_bounds(p->d_res, d_bounds, st), "bounds export");
    return FO_OK;
}

fo_status fo_chebyshev_coeffs(fo_ctx* ctx, double kT, double mu, double emin, double emax,
                              int32_t n_terms, int32_t n_quad, double* d_c, void* stream) {
    if (!ctx) return FO_ERR_ARG;
    if (!d_c || n_terms < 1 || n_terms > 4096) return fail(ctx, FO_ERR_ARG, "bad n_terms or output");
    if (!(kT > 0.0) || !(emax > emin)) return fail(ctx, FO_ERR_ARG, "need kT > 0 and emax > emin");
    const int M = n_quad > 0 ? n_quad : (2048 > 4 * n_terms ? 2048 : 4 * n_terms);
    if (M < n_terms) return fail(ctx, FO_ERR_ARG, "n_quad must be >= n_terms");
    DeviceGuard g(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PlanKey key;
    key.n = {1};
    key.mode = MODE_COEFFS;
    key.n_terms = n_terms;
    key.n_quad = n_quad;
    Plan* p = nullptr;
    FO_TRY(get_plan(ctx, key, &p));
    InstIO io;
    std::memset(&io, 0, sizeof(io));
    io.kT = kT;
    io.mu = mu;
    io.emin = emin;
    io.emax = emax;
    FO_CUDA(launch_set_io(&io, 1, p->d_io, p->d_inst, 0, st), "set_io");
    FO_CUDA(launch_bounds(p->d_inst, p->d_io, 1, p->wg.dev, p->part_g, 1, st), "bounds");
    FO_CUDA(launch_set_mu(p->d_inst, p->d_io, 1, st), "mu");
    FO_CUDA(launch_coefficients(p->d_inst, p->d_io, 1, p->sh, p->ct, 0, st, nullptr), "coeffs");
    FO_CUDA(cudaMemcpyAsync(d_c, p->inst[0].c, 8 * (size_t)n_terms, cudaMemcpyDeviceToDevice, st), "copy");
    return FO_OK;
}

fo_status fo_density_matrix(fo_ctx* ctx, const double* dH, int64_t n, int64_t ld, double n_e,
                            const fo_params* params, double* dP, int64_t ldp, fo_result* res, void* stream) {
    if (!ctx) return FO_ERR_ARG;
    DeviceGuard g(ctx->device);
    double* P = dP;
    return density_batch(ctx, 1, &dH, &n, &ld, &n_e, nullptr, params, &P, &ldp, res,
                         reinterpret_cast<cudaStream_t>(stream));
}

fo_status fo_density_matrix_batched(fo_ctx* ctx, int32_t batch, const double* const* dH, const int64_t* n,
                                    const int64_t* ld, const double* n_e, const double* kT,
                                    const fo_params* params, double* const* dP, const int64_t* ldp,
                                    fo_result* res, void* stream) {
    if (!ctx) return FO_ERR_ARG;
    DeviceGuard g(ctx->device);
    return density_batch(ctx, batch, dH, n, ld, n_e, kT, params, dP, ldp, res,
                         reinterpret_cast<cudaStream_t>(stream));
}

fo_status fo_density_matrix_batched_host(fo_ctx* ctx, int32_t batch, const double* const* hH, const int64_t* n,
                                         const int64_t* ld, const double* n_e, const double* kT,
                                         const fo_params* params, double* const* hP, const int64_t* ldp,
                                         fo_result* res, void* stream) {
    if (!ctx) return FO_ERR_ARG;
    if (batch < 1 || !hH || !hP || !n || !n_e || !params) return fail(ctx, FO_ERR_ARG, "bad arguments");
    for (int b = 0; b < batch; ++b)
        if (!hH[b] || !hP[b] || n[b] < 1 || (ld && ld[b] < n[b]) || (ldp && ldp[b] < n[b]))
            return fail(ctx, FO_ERR_ARG, "bad instance arguments");
    DeviceGuard g(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool async = (params->flags & FO_FLAG_NO_RESULT_SYNC) != 0;
    if (!ctx->h2d) {
        FO_CUDA(cudaStreamCreateWithFlags(&ctx->h2d, cudaStreamNonBlocking), "copy stream");
        FO_CUDA(cudaStreamCreateWithFlags(&ctx->d2h, cudaStreamNonBlocking), "copy stream");
        for (auto& hs : ctx->hslot)
            for (cudaEvent_t* e : {&hs.in, &hs.done, &hs.out})
                FO_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "copy event");
    }
    fo_ctx::HostSlot& hs = ctx->hslot[ctx->hnext];
    ctx->hnext ^= 1;
    // device staging: H and P of every instance, densely packed
    std::vector<size_t> off(batch);
    size_t total = 0;
    for (int b = 0; b < batch; ++b) {
        off[b] = total;
        total += 2 * align256((size_t)n[b] * n[b] * 8);
    }
    if (hs.bytes < total) {
        if (hs.buf) {
            FO_CUDA(cudaEventSynchronize(hs.out), "staging slot");
            cudaFree(hs.buf);
            hs.buf = nullptr;
            hs.bytes = 0;
        }
        if (cudaMalloc(&hs.buf, total) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, FO_ERR_NOMEM, "staging allocation failed");
        }
        hs.bytes = total;
        hs.used = false;
    }
    // the slot's previous outputs have left (and its previous solve has finished) before its
    // inputs are overwritten
    if (hs.used) FO_CUDA(cudaStreamWaitEvent(ctx->h2d, hs.out, 0), "slot wait");
    std::vector<const double*> dH(batch);
    std::vector<double*> dP(batch);
    std::vector<int64_t> ldn(n, n + batch);
    char* base = reinterpret_cast<char*>(hs.buf);
    for (int b = 0; b < batch; ++b) {
        double* h = reinterpret_cast<double*>(base + off[b]);
        dH[b] = h;
        dP[b] = reinterpret_cast<double*>(base + off[b] + align256((size_t)n[b] * n[b] * 8));
        const int64_t l = ld ? ld[b] : n[b];
        if (l == n[b])   // contiguous rows: one linear copy
            FO_CUDA(cudaMemcpyAsync(h, hH[b], (size_t)n[b] * n[b] * 8, cudaMemcpyHostToDevice, ctx->h2d), "H2D");
        else
            FO_CUDA(cudaMemcpy2DAsync(h, n[b] * 8, hH[b], l * 8, n[b] * 8, n[b], cudaMemcpyHostToDevice, ctx->h2d),
                    "H2D");
    }
    FO_CUDA(cudaEventRecord(hs.in, ctx->h2d), "copy event");
    FO_CUDA(cudaStreamWaitEvent(st, hs.in, 0), "inputs wait");
    fo_params prm = *params;
    if (!async) prm.flags &= ~FO_FLAG_NO_RESULT_SYNC;
    std::vector<fo_result> local(batch);
    fo_status s = density_batch(ctx, batch, dH.data(), n, ldn.data(), n_e, kT, &prm, dP.data(), ldn.data(),
                                res ? res : local.data(), st);
    if (s != FO_OK && s != FO_ERR_NOT_CONVERGED) return s;
    FO_CUDA(cudaEventRecord(hs.done, st), "solve event");
    FO_CUDA(cudaStreamWaitEvent(ctx->d2h, hs.done, 0), "solve wait");
    for (int b = 0; b < batch; ++b) {
        const int64_t l = ldp ? ldp[b] : n[b];
        if (l == n[b])
            FO_CUDA(cudaMemcpyAsync(hP[b], dP[b], (size_t)n[b] * n[b] * 8, cudaMemcpyDeviceToHost, ctx->d2h), "D2H");
        else
            FO_CUDA(cudaMemcpy2DAsync(hP[b], l * 8, dP[b], n[b] * 8, n[b] * 8, n[b], cudaMemcpyDeviceToHost,
                                      ctx->d2h),
                    "D2H");
    }
    FO_CUDA(cudaEventRecord(hs.out, ctx->d2h), "copy event");
    hs.used = true;
    if (!async) FO_CUDA(cudaEventSynchronize(hs.out), "sync");
    return s;
}

fo_status fo_host_wait(fo_ctx* ctx) {
    if (!ctx) return FO_ERR_ARG;
    DeviceGuard g(ctx->device);
    for (auto& hs : ctx->hslot)
        if (hs.used) FO_CUDA(cudaEventSynchronize(hs.out), "host wait");
    int flag = 0;
    FO_CUDA(cudaMemcpy(&flag, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost), "flag readback");
    if (flag) return fail(ctx, FO_ERR_DEVICE_TIMEOUT, "a kernel gave up a bounded wait");
    return FO_OK;
}

fo_status fo_density_matrix_host(fo_ctx* ctx, const double* hH, int64_t n, int64_t ld, double n_e,
                                 const fo_params* params, double* hP, int64_t ldp, fo_result* res,
                                 void* stream) {
    if (!ctx) return FO_ERR_ARG;
    if (!hH || !hP || n < 1 || ld < n || ldp < n || !params) return fail(ctx, FO_ERR_ARG, "bad arguments");
    double* P = hP;
    return fo_density_matrix_batched_host(ctx, 1, &hH, &n, &ld, &n_e, nullptr, params, &P, &ldp, res, stream);
}

fo_status fo_moments(fo_ctx* ctx, const double* dH, int64_t n, int64_t ld, const double* d_bounds,
                     int32_t n_moments, int32_t precision, double* d_tau, void* stream) {
    if (!ctx) return FO_ERR_ARG;
    if (!dH || !d_bounds || !d_tau || n < 1 || ld < n || n_moments < 1 || n_moments > 256)
        return fail(ctx, FO_ERR_ARG, "bad arguments");
    DeviceGuard g(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int K = n_moments <= 2 ? 1 : (n_moments + 1) / 2;
    // k = K baby steps, m = 2: the assembly then covers tau_0 .. tau_{2K-1}
    PlanKey key;
    key.n = {n};
    key.mode = MODE_MOMENTS;
    key.n_terms = 2 * K;
    key.k_req = K;
    key.prec = precision;
    key.use_given = 1;
    Plan* p = nullptr;
    FO_TRY(get_plan(ctx, key, &p));
    InstIO io;
    std::memset(&io, 0, sizeof(io));
    io.H = dH;
    io.ldh = ld;
    io.bounds_src = d_bounds;
    Run run;
    FO_CUDA(launch_set_io(&io, 1, p->d_io, p->d_inst, 0, st), "set_io");
    FO_CUDA(launch_bounds(p->d_inst, p->d_io, 1, p->wg.dev, p->part_g, 1, st), "bounds");
    FO_CUDA(launch_scale(p->d_inst, p->d_io, p->wsc.dev, p->sh, st, ctx->flag + 1), "scale");
    FO_TRY(baby_steps(ctx, *p, p->sh.k, st, &run));
    FO_TRY(exact_moments(ctx, *p, st, &run));
    FO_CUDA(cudaMemcpyAsync(d_tau, p->inst[0].tau, 8 * (size_t)n_moments, cudaMemcpyDeviceToDevice, st),
            "tau copy");
    return FO_OK;
}

fo_status fo_profile_enable(fo_ctx* ctx, int32_t enable) {
    if (!ctx) return FO_ERR_ARG;
    DeviceGuard g(ctx->device);
    prof_collect(ctx);
    for (int i = 0; i < FO_PROFILE_STAGES; ++i) {
        ctx->prof_ms[i] = 0.0;
        ctx->prof_flops[i] = 0.0;
        ctx->prof_launches[i] = 0;
    }
    ctx->prof_calls = 0;
    ctx->prof = enable != 0;
    return FO_OK;
}

fo_status fo_profile_read(fo_ctx* ctx, fo_profile* out, int32_t reset) {
    if (!ctx || !out) return FO_ERR_ARG;
    DeviceGuard g(ctx->device);
    prof_collect(ctx);
    for (int i = 0; i < FO_PROFILE_STAGES; ++i) {
        out->ms[i] = ctx->prof_ms[i];
        out->flops[i] = ctx->prof_flops[i];
        out->launches[i] = ctx->prof_launches[i];
    }
    out->calls = ctx->prof_calls;
    if (reset) {
        for (int i = 0; i < FO_PROFILE_STAGES; ++i) {
            ctx->prof_ms[i] = 0.0;
            ctx->prof_flops[i] = 0.0;
            ctx->prof_launches[i] = 0;
        }
        ctx->prof_calls = 0;
    }
    return FO_OK;
}

fo_status fo_recurrence_product(fo_ctx* ctx, int32_t precision, int32_t symmetric, int64_t n, int64_t ld,
                                const float* dA, const float* dB, const float* dC, const float* dD,
                                float alpha, float beta, float shift, float* dOut, void* stream) {
    if (!ctx) return FO_ERR_ARG;
    if (precision == FO_PREC_FP64 || tc_planes(precision) == 0)
        return fail(ctx, FO_ERR_ARG, "precision must be a split form");
    if (!dA || !dB || !dOut || n < 1 || ld < n || n > 65536) return fail(ctx, FO_ERR_ARG, "bad arguments");
    DeviceGuard g(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PlanKey key;
    key.n = {n};
    key.mode = MODE_PRODUCT;
    key.prec = precision;
    key.sym = symmetric ? 1 : 0;
    key.n_terms = 4;
    key.k_req = 2;
    Plan* p = nullptr;
    FO_TRY(get_plan(ctx, key, &p));
    const Inst& in = p->inst[0];
    const Shape& sh = p->sh;
    const float ps = sh.fp16 ? sh.pscale_t : 1.0f;
    InstIO io;
    std::memset(&io, 0, sizeof(io));
    FO_CUDA(launch_set_io(&io, 1, p->d_io, p->d_inst, 0, st), "set_io");
    // slots: 0 = A, 1 = B, 2 = C, 3 = D, 4 = out
    FO_CUDA(launch_pack_f32(dA, n, ld, in.slots, in.np, sh.planes, sh.fp16, ps, st), "pack");
    FO_CUDA(launch_pack_f32(dB, n, ld, in.slots + in.slot_bytes, in.np, sh.planes, sh.fp16, ps, st), "pack");
    if (dC) FO_CUDA(launch_pack_f32(dC, n, ld, in.slots + 2 * in.slot_bytes, in.np, 0, 0, 1.0f, st), "pack");
    if (dD) FO_CUDA(launch_pack_f32(dD, n, ld, in.slots + 3 * in.slot_bytes, in.np, 0, 0, 1.0f, st), "pack");
    Step stp = make_step(*p, 0, 1, dC ? 2 : -1, dD ? 3 : -1, 4, alpha, beta, shift, false, false, false, false, ctx);
    stp.planes = 0;
    stp.lower_master = 1;   // the whole float32 result is copied out
    Run run;
    FO_TRY(run_product(ctx, *p, stp, st, "product", 0, &run));
    FO_CUDA(cudaMemcpy2DAsync(dOut, ld * 4, in.slots + 4 * in.slot_bytes, in.np * 4, n * 4, n,
                              cudaMemcpyDeviceToDevice, st),
            "copy out");
    return FO_OK;
}

fo_status fo_learned_features(fo_ctx* ctx, int32_t batch, const double* const* dH, const int64_t* n,
                              const int64_t* ld, const double* n_e, const double* kT, const fo_params* params,
                              float* d_feat, float* d_target, fo_result* res, void* stream) {
    if (!ctx) return FO_ERR_ARG;
    DeviceGuard g(ctx->device);
    return features_batch(ctx, batch, dH, n, ld, n_e, kT, params, d_feat, d_target, res,
                          reinterpret_cast<cudaStream_t>(stream));
}

fo_status fo_mlp_init(fo_ctx* ctx, uint64_t seed) {
    if (!ctx) return FO_ERR_ARG;
    DeviceGuard g(ctx->device);
    std::vector<float> prm, norm;
    init_host_params(seed, prm, norm);
    return upload_model(ctx, prm.data(), norm.data());
}

fo_status fo_mlp_set_params(fo_ctx* ctx, const float* h_params, const float* h_norm) {
    if (!ctx || !h_params) return FO_ERR_ARG;
    DeviceGuard g(ctx->device);
    std::vector<float> prm, norm;
    init_host_params(0, prm, norm);
    return upload_model(ctx, h_params, h_norm ? h_norm : norm.data());
}

fo_status fo_mlp_get_params(fo_ctx* ctx, float* h_params, float* h_norm) {
    if (!ctx) return FO_ERR_ARG;
    if (!ctx->mlp) return fail(ctx, FO_ERR_UNSUPPORTED, "no model");
    DeviceGuard g(ctx->device);
    if (h_params && cudaMemcpy(h_params, mlp_params(ctx), sizeof(float) * mlp_offsets().total,
                               cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(ctx, FO_ERR_CUDA, "model download failed");
    if (h_norm && cudaMemcpy(h_norm, mlp_norm(ctx), sizeof(float) * kMlpNorm, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(ctx, FO_ERR_CUDA, "model download failed");
    return FO_OK;
}

fo_status fo_mlp_forward(fo_ctx* ctx, const float* d_x, int32_t n, float* d_y, void* stream) {
    if (!ctx || !d_x || !d_y || n < 1) return ctx ? fail(ctx, FO_ERR_ARG, "bad arguments") : FO_ERR_ARG;
    if (!ctx->mlp_ready) return fail(ctx, FO_ERR_UNSUPPORTED, "no model");
    DeviceGuard g(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    FO_TRY(ensure_mlp_scratch(ctx, (size_t)n * 4 * kMlpHidden));
    float* z1 = ctx->mlp_scratch;
    float* a1 = z1 + (size_t)n * kMlpHidden;
    float* z2 = a1 + (size_t)n * kMlpHidden;
    float* a2 = z2 + (size_t)n * kMlpHidden;
    FO_CUDA(mlp_forward(mlp_params(ctx), d_x, n, z1, a1, z2, a2, d_y, st), "network");
    return FO_OK;
}

fo_status fo_mlp_gradients(fo_ctx* ctx, const float* d_x, const float* d_t, int32_t n, float* d_grad,
                           float* h_loss, void* stream) {
    if (!ctx || !d_x || !d_t || !d_grad || n < 1) return ctx ? fail(ctx, FO_ERR_ARG, "bad arguments") : FO_ERR_ARG;
    if (!ctx->mlp_ready) return fail(ctx, FO_ERR_UNSUPPORTED, "no model");
    DeviceGuard g(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t B = (size_t)n;
    FO_TRY(ensure_mlp_scratch(ctx, B * (6 * kMlpHidden + 2 * kMlpOut) + 1));
    float* z1 = ctx->mlp_scratch;
    float* a1 = z1 + B * kMlpHidden;
    float* z2 = a1 + B * kMlpHidden;
    float* a2 = z2 + B * kMlpHidden;
    float* dz2 = a2 + B * kMlpHidden;
    float* dz1 = dz2 + B * kMlpHidden;
    float* y = dz1 + B * kMlpHidden;
    float* dy = y + B * kMlpOut;
    float* loss = dy + B * kMlpOut;
    FO_CUDA(mlp_forward(mlp_params(ctx), d_x, n, z1, a1, z2, a2, y, st), "network");
    FO_CUDA(mlp_backward(mlp_params(ctx), d_x, d_t, n, z1, a1, z2, a2, y, dy, dz2, dz1, d_grad, loss, st),
            "backward");
    if (h_loss) {
        FO_CUDA(cudaMemcpyAsync(h_loss, loss, sizeof(float), cudaMemcpyDeviceToHost, st), "loss");
        FO_CUDA(cudaStreamSynchronize(st), "sync");
    }
    return FO_OK;
}

fo_status fo_mlp_train(fo_ctx* ctx, const float* d_feat, const float* d_target, int32_t n, int32_t epochs,
                       int32_t batch, float lr, uint64_t seed, float* h_loss, void* stream) {
    if (!ctx) return FO_ERR_ARG;
    if (!d_feat || !d_target || n < 2 || epochs < 1 || batch < 1 || !(lr > 0.0f))
        return fail(ctx, FO_ERR_ARG, "bad training arguments");
    DeviceGuard g(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!ctx->mlp_ready) FO_TRY(fo_mlp_init(ctx, seed));
    const int B = batch < n ? batch : n;
    const int steps = (n + B - 1) / B;
    const size_t total_steps = (size_t)steps * epochs;
    const size_t Bz = (size_t)B;
    const size_t need = Bz * (kMlpIn + kMlpOut + 6 * kMlpHidden + 2 * kMlpOut) + total_steps + (size_t)n;
    FO_TRY(ensure_mlp_scratch(ctx, need));
    float* xb = ctx->mlp_scratch;
    float* tb = xb + Bz * kMlpIn;
    float* z1 = tb + Bz * kMlpOut;
    float* a1 = z1 + Bz * kMlpHidden;
    float* z2 = a1 + Bz * kMlpHidden;
    float* a2 = z2 + Bz * kMlpHidden;
    float* dz2 = a2 + Bz * kMlpHidden;
    float* dz1 = dz2 + Bz * kMlpHidden;
    float* y = dz1 + Bz * kMlpHidden;
    float* dy = y + Bz * kMlpOut;
    float* losses = dy + Bz * kMlpOut;
    int* idx = reinterpret_cast<int*>(losses + total_steps);
    float* norm = mlp_norm(ctx);
    // normalisation from the training set
    FO_CUDA(mlp_col_stats(d_feat, n, kMlpIn, norm, norm + kMlpIn, st), "stats");
    FO_CUDA(mlp_col_stats(d_target, n, kMlpOut, norm + 2 * kMlpIn, norm + 2 * kMlpIn + kMlpOut, st), "stats");
    const int P = mlp_offsets().total;
    std::vector<int> perm(n);
    uint64_t rs = seed ^ 0x5DEECE66Dull;
    size_t step_i = 0;
    for (int e = 0; e < epochs; ++e) {
        std::iota(perm.begin(), perm.end(), 0);
        for (int q = n - 1; q > 0; --q) {   // Fisher-Yates
            const int r = (int)(splitmix64(rs) % (uint64_t)(q + 1));
            std::swap(perm[q], perm[r]);
        }
        FO_CUDA(cudaStreamSynchronize(st), "sync");
        FO_CUDA(cudaMemcpy(idx, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice), "order");
        for (int j = 0; j < steps; ++j, ++step_i) {
            const int Bj = (j + 1) * B <= n ? B : n - j * B;
            FO_CUDA(mlp_gather_norm(d_feat, idx + j * B, Bj, kMlpIn, norm, norm + kMlpIn, xb, st), "batch");
            FO_CUDA(mlp_gather_norm(d_target, idx + j * B, Bj, kMlpOut, norm + 2 * kMlpIn,
                                    norm + 2 * kMlpIn + kMlpOut, tb, st),
                    "batch");
            FO_CUDA(mlp_forward(mlp_params(ctx), xb, Bj, z1, a1, z2, a2, y, st), "network");
            FO_CUDA(mlp_backward(mlp_params(ctx), xb, tb, Bj, z1, a1, z2, a2, y, dy, dz2, dz1, mlp_grad(ctx),
                                 losses + step_i, st),
                    "backward");
            ctx->mlp_step += 1;
            FO_CUDA(mlp_adam(mlp_params(ctx), mlp_grad(ctx), mlp_m(ctx), mlp_v(ctx), P, lr, ctx->mlp_step, st),
                    "adam");
        }
    }
    std::vector<float> hl(total_steps);
    FO_CUDA(cudaStreamSynchronize(st), "sync");
    FO_CUDA(cudaMemcpy(hl.data(), losses, sizeof(float) * total_steps, cudaMemcpyDeviceToHost), "losses");
    if (h_loss)
        for (int e = 0; e < epochs; ++e) {
            double a = 0.0;
            for (int j = 0; j < steps; ++j) a += hl[(size_t)e * steps + j];
            h_loss[e] = (float)(a / steps);
        }
    ctx->mlp_ready = true;
    return FO_OK;
}

fo_status fo_mlp_save(fo_ctx* ctx, const char* path) {
    if (!ctx || !path) return FO_ERR_ARG;
    if (!ctx->mlp_ready) return fail(ctx, FO_ERR_UNSUPPORTED, "no model");
    const int P = mlp_offsets().total;
    std::vector<float> prm(P), norm(kMlpNorm);
    FO_TRY(fo_mlp_get_params(ctx, prm.data(), norm.data()));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(ctx, FO_ERR_ARG, std::string("cannot write ") + path);
    const char magic[8] = {'F', 'O', 'M', 'L', 'P', '1', 0, 0};
    const int32_t dims[5] = {kMlpIn, kMlpHidden, kMlpOut, P, kMlpNorm};
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(dims, sizeof(int32_t), 5, f) == 5 &&
              std::fwrite(norm.data(), sizeof(float), kMlpNorm, f) == (size_t)kMlpNorm &&
              std::fwrite(prm.data(), sizeof(float), P, f) == (size_t)P;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? FO_OK : fail(ctx, FO_ERR_ARG, std::string("write failed: ") + path);
}

fo_status fo_mlp_load(fo_ctx* ctx, const char* path) {
    if (!ctx || !path) return FO_ERR_ARG;
    DeviceGuard g(ctx->device);
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(ctx, FO_ERR_ARG, std::string("cannot read ") + path);
    char magic[8];
    int32_t dims[5];
    const int P = mlp_offsets().total;
    std::vector<float> prm(P), norm(kMlpNorm);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "FOMLP1", 6) == 0 &&
              std::fread(dims, sizeof(int32_t), 5, f) == 5 && dims[0] == kMlpIn && dims[1] == kMlpHidden &&
              dims[2] == kMlpOut && dims[3] == P && dims[4] == kMlpNorm &&
              std::fread(norm.data(), sizeof(float), kMlpNorm, f) == (size_t)kMlpNorm &&
              std::fread(prm.data(), sizeof(float), P, f) == (size_t)P;
    std::fclose(f);
    if (!ok) return fail(ctx, FO_ERR_ARG, std::string("not a model file of this layout: ") + path);
    return upload_model(ctx, prm.data(), norm.data());
}

}  // extern "C"
