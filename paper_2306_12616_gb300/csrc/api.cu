// C ABI of the solver (include/fermi.h) and the host orchestration of one density matrix.
//
// The host only plans (k, m, padding, workspace layout), checks arguments and enqueues
// kernels; every number of the method is computed on the device, and the whole sequence
// runs on the caller's stream without host synchronisation until the optional readback of
// the scalar results.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace fo;

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
    void* ws = nullptr;        // device workspace
    size_t ws_bytes = 0;
    void* stage = nullptr;     // device staging for the host-buffer entry point
    size_t stage_bytes = 0;
    DevResult* res = nullptr;  // device result record (own allocation)
    int* flag = nullptr;       // tensor-core wait-timeout flag
};

namespace {

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

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

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

#define FO_CUDA(call, where)                                          \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ == cudaSuccess && debug_sync()) e_ = cudaDeviceSynchronize(); \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where);      \
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

// Starts a timed stage when profiling is on; returns a handle for prof_end (or -1).
int prof_begin(fo_ctx* ctx, cudaStream_t st, int stage) {
    if (!ctx->prof) return -1;
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

fo_status ensure_ws(fo_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return FO_OK;
    if (ctx->ws) {
        cudaDeviceSynchronize();
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    if (cudaMalloc(&ctx->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, FO_ERR_NOMEM, "workspace allocation of " + std::to_string(bytes) + " bytes failed");
    }
    // the zero border of every padded matrix is relied upon; clear once
    if (cudaMemset(ctx->ws, 0, bytes) != cudaSuccess) return fail(ctx, FO_ERR_CUDA, "workspace clear failed");
    ctx->ws_bytes = bytes;
    return FO_OK;
}

// --------------------------------------------------------------------------- plan
struct Plan {
    int64_t n = 0, np = 0;
    int n_terms = 0, k = 0, m = 0, km = 0, M = 0;
    int prec = 0, planes = 0, fp16 = 0;
    bool giants = false;       // giant steps T_{lk} for exact moments
    bool moments = false;      // compute tau
    size_t slot_bytes = 0;
    int n_tslots = 0;          // T_1..T_k (+ giants)
    size_t off_t = 0, off_r = 0;
    size_t off_c = 0, off_g = 0, off_tau = 0, off_w = 0, off_f = 0, off_ct = 0;
    size_t off_diag = 0, off_gram = 0, off_gpart = 0, off_part = 0;
    int gram_nblocks = 0, nparts = 0;
    size_t total = 0;
    float pscale_t = 1.0f;     // fp16 plane scale of T and giant slots
    float pscale_r = 1.0f;     // fp16 plane scale of R / Clenshaw slots
};

bool plan_km(int n_terms, int k_req, int* k, int* m) {
    if (n_terms < 1) return false;
    int kk = k_req > 0 ? k_req : (int)std::ceil(std::sqrt((double)n_terms));
    if (kk < 1) kk = 1;
    *k = kk;
    *m = (n_terms + kk - 1) / kk;
    return true;
}

fo_status make_plan(fo_ctx* ctx, int64_t n, int n_terms, int k_req, int prec, bool giants,
                    bool moments, int n_quad, Plan* p) {
    if (n < 1) return fail(ctx, FO_ERR_ARG, "n must be >= 1");
    if (n > 65536) return fail(ctx, FO_ERR_ARG, "n above 65536 is not supported");
    if (n_terms < 1 || n_terms > 4096) return fail(ctx, FO_ERR_ARG, "n_terms must be in [1, 4096]");
    if (prec < FO_PREC_FP64 || prec > FO_PREC_BF16X1) return fail(ctx, FO_ERR_ARG, "unknown precision");
    p->n = n;
    p->np = ((n + kPad - 1) / kPad) * kPad;
    // tensor-core tiles are 128 x 256: keep at least one full column tile
    if (prec != FO_PREC_FP64 && p->np < 256) p->np = 256;
    p->n_terms = n_terms;
    if (!plan_km(n_terms, k_req, &p->k, &p->m)) return fail(ctx, FO_ERR_ARG, "bad k");
    if (p->k > 64 || p->m > 64) return fail(ctx, FO_ERR_ARG, "k and m must not exceed 64");
    p->km = p->k * p->m;
    p->M = n_quad > 0 ? n_quad : (2048 > 4 * n_terms ? 2048 : 4 * n_terms);
    if (p->M < n_terms) return fail(ctx, FO_ERR_ARG, "n_quad must be >= n_terms");
    p->prec = prec;
    p->planes = tc_planes(prec);
    p->fp16 = prec == FO_PREC_FP16X2;
    p->giants = giants && p->m > 2;
    if (moments && p->k > 33) return fail(ctx, FO_ERR_UNSUPPORTED, "exact moments support k <= 33");
    p->moments = moments;
    const size_t np2 = (size_t)p->np * (size_t)p->np;
    p->slot_bytes = prec == FO_PREC_FP64 ? align256(np2 * 8) : align256(np2 * 4 + p->planes * np2 * 2);
    p->n_tslots = p->k + (p->giants ? p->m - 2 : 0);
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += align256(b); return o; };
    p->off_t = take(p->slot_bytes * p->n_tslots);
    p->off_r = take(p->slot_bytes * p->m);
    p->off_c = take(8 * (size_t)p->km);
    p->off_g = take(8 * (size_t)p->km);
    p->off_tau = take(8 * (size_t)(p->km + 2));
    p->off_w = take(8 * (size_t)p->M);
    p->off_f = take(8 * (size_t)p->M);
    p->off_ct = take(8 * 4 * (size_t)p->M);
    p->off_diag = take(8 * (size_t)(p->k + p->m + 2));
    const int npairs = (p->m > 1 ? p->m - 1 : 1) * p->k;
    p->off_gram = take(8 * (size_t)npairs);
    p->gram_nblocks = gram_blocks(p->np, p->m - 1, p->k);
    p->off_gpart = take(8 * (size_t)npairs * p->gram_nblocks);
    p->nparts = 2 * (ctx->num_sms > 0 ? ctx->num_sms : 152);
    p->off_part = take(8 * 3 * (size_t)p->nparts + 64);
    p->total = off;
    // fp16 planes hold v * scale; T slots have |entries| <= 1 (spectrum of X in [-1, 1])
    p->pscale_t = 256.0f;
    p->pscale_r = 1.0f;
    return FO_OK;
}

char* wsb(fo_ctx* ctx) { return reinterpret_cast<char*>(ctx->ws); }

struct Slots {
    char* t;     // T_1 .. T_k, giants
    char* r;     // R_0 .. R_{m-1}
    size_t stride;
    int64_t np;
    int planes;
    MatF32 mat(char* base, int i) const {
        MatF32 x;
        x.x = reinterpret_cast<float*>(base + stride * i);
        x.planes = reinterpret_cast<uint16_t*>(base + stride * i + (size_t)np * np * 4);
        x.ld = np;
        x.plane_stride = np * np;
        return x;
    }
    MatF32 T(int i) const { return mat(t, i); }      // slot index
    MatF32 R(int l) const { return mat(r, l); }
    double* Td(int i) const { return reinterpret_cast<double*>(t + stride * i); }
    double* Rd(int l) const { return reinterpret_cast<double*>(r + stride * l); }
};

// Slot of T_{j k} for j >= 1: T_k is baby slot k-1, giants T_{2k}.. follow.
int giant_slot(const Plan& p, int j) { return j == 1 ? p.k - 1 : p.k + j - 2; }

// One recurrence product out = alpha A B + beta C + D + shift I in the plan's arithmetic.
struct Product {
    int a, b;            // operand slots (tbase / rbase chosen by flags)
    bool a_r = false, b_r = false;
    int c = -1, d = -1;  // -1 = absent
    bool c_r = false, d_r = false;
    int out = -1;
    bool out_r = false;
    double alpha = 1, beta = 0, shift = 0;
    double* out64 = nullptr;
    int64_t ldo = 0;
    const char* tag = "product";  // stage name for error messages
    int index = 0;
};

fo_status run_product_impl(fo_ctx* ctx, const Plan& p, const Slots& S, const Product& q,
                           cudaStream_t st, int sym);

// Algorithmic flops of one symmetric product: n^2 (n+1) per split product.
double product_flops(const Plan& p) {
    const double n = (double)p.n;
    const int s = p.prec == FO_PREC_BF16X3 ? 6 : (p.prec == FO_PREC_FP16X2 ? 3 : 1);
    return s * n * n * (n + 1.0);
}

fo_status run_product(fo_ctx* ctx, const Plan& p, const Slots& S, const Product& q, cudaStream_t st,
                      int sym) {
    const int h = prof_begin(ctx, st, FO_STAGE_PRODUCTS);
    fo_status r = run_product_impl(ctx, p, S, q, st, sym);
    prof_end(ctx, st, h, product_flops(p), 1);
    return r;
}

fo_status run_product_impl(fo_ctx* ctx, const Plan& p, const Slots& S, const Product& q,
                           cudaStream_t st, int sym) {
    if (p.prec == FO_PREC_FP64) {
        const double* A = q.a_r ? S.Rd(q.a) : S.Td(q.a);
        const double* B = q.b_r ? S.Rd(q.b) : S.Td(q.b);
        const double* C = q.c < 0 ? nullptr : (q.c_r ? S.Rd(q.c) : S.Td(q.c));
        const double* D = q.d < 0 ? nullptr : (q.d_r ? S.Rd(q.d) : S.Td(q.d));
        double* out = q.out < 0 ? nullptr : (q.out_r ? S.Rd(q.out) : S.Td(q.out));
        FO_CUDA(launch_gemm_f64(A, B, p.np, q.alpha, C, q.beta, D, q.shift, (int)p.n, out, q.out64,
                                q.ldo, st),
                "gemm_f64");
        return FO_OK;
    }
    const MatF32 A = q.a_r ? S.R(q.a) : S.T(q.a);
    const MatF32 B = q.b_r ? S.R(q.b) : S.T(q.b);
    Epilogue ep;
    std::memset(&ep, 0, sizeof(ep));
    const float sa = p.fp16 ? (q.a_r ? p.pscale_r : p.pscale_t) : 1.0f;
    const float sb = p.fp16 ? (q.b_r ? p.pscale_r : p.pscale_t) : 1.0f;
    ep.alpha = (float)(q.alpha / ((double)sa * sb));
    ep.beta = (float)q.beta;
    ep.shift = (float)q.shift;
    ep.n_real = (int32_t)p.n;
    ep.C = q.c < 0 ? nullptr : (q.c_r ? S.R(q.c).x : S.T(q.c).x);
    ep.D = q.d < 0 ? nullptr : (q.d_r ? S.R(q.d).x : S.T(q.d).x);
    ep.ld = p.np;
    if (q.out >= 0) {
        ep.out = q.out_r ? S.R(q.out) : S.T(q.out);
        ep.planes = p.planes;
        ep.plane_scale = q.out_r ? p.pscale_r : p.pscale_t;
    }
    ep.out64 = q.out64;
    ep.ldo = q.ldo;
    ep.fp16 = p.fp16;
    ep.dbg = ctx->flag + 1;
    std::string err;
    cudaError_t e = tc_gemm(p.prec, p.np, A, B, ep, sym, ctx->flag, st, &err);
    if (e == cudaSuccess && debug_sync()) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        const std::string where = std::string("tc_gemm ") + q.tag + " " + std::to_string(q.index);
        if (!err.empty()) return fail(ctx, FO_ERR_CUDA, where + ": " + err);
        return cuda_fail(ctx, e, where.c_str());
    }
    return FO_OK;
}

#define FO_TRY(x)                      \
    do {                               \
        fo_status s_ = (x);            \
        if (s_ != FO_OK) return s_;    \
    } while (0)

// Scale H into slot T_1 (float64, or float32 + planes).
fo_status pack_x(fo_ctx* ctx, const Plan& p, const Slots& S, const double* dH, int64_t ld,
                 cudaStream_t st) {
    if (p.prec == FO_PREC_FP64)
        FO_CUDA(launch_scale_f64(dH, p.n, ld, ctx->res, S.Td(0), p.np, st, ctx->flag + 1), "scale");
    else
        FO_CUDA(launch_scale_split(dH, p.n, ld, ctx->res, S.T(0), p.np, p.planes, p.fp16, p.pscale_t, st,
                                   ctx->flag + 1),
                "scale_split");
    return FO_OK;
}

// Baby steps T_2..T_k: T_{i+1} = 2 T_1 T_i - T_{i-1} (T_0 = I as a diagonal shift).
fo_status baby_steps(fo_ctx* ctx, const Plan& p, const Slots& S, int kmax, cudaStream_t st,
                     int sym, int* n_gemm) {
    for (int i = 1; i < kmax; ++i) {
        Product q;
        q.a = 0;
        q.b = i - 1;
        q.out = i;
        q.alpha = 2.0;
        q.tag = "baby";
        q.index = i + 1;
        if (i == 1) { q.shift = -1.0; }
        else { q.c = i - 2; q.beta = -1.0; }
        FO_TRY(run_product(ctx, p, S, q, st, sym));
        ++*n_gemm;
    }
    return FO_OK;
}

// Giant steps T_{2k}..T_{(m-1)k}: T_{(j+1)k} = 2 T_k T_{jk} - T_{(j-1)k}.
fo_status giant_steps(fo_ctx* ctx, const Plan& p, const Slots& S, cudaStream_t st, int sym,
                      int* n_gemm) {
    for (int j = 1; j + 1 <= p.m - 1; ++j) {
        Product q;
        q.a = giant_slot(p, 1);
        q.b = giant_slot(p, j);
        q.out = giant_slot(p, j + 1);
        q.alpha = 2.0;
        q.tag = "giant";
        q.index = j + 1;
        if (j == 1) { q.shift = -1.0; }
        else { q.c = giant_slot(p, j - 1); q.beta = -1.0; }
        FO_TRY(run_product(ctx, p, S, q, st, sym));
        ++*n_gemm;
    }
    return FO_OK;
}

// Exact moments tau_0..tau_{n_terms-1} (needs the giant steps).
fo_status exact_moments(fo_ctx* ctx, const Plan& p, const Slots& S, cudaStream_t st) {
    const int is64 = p.prec == FO_PREC_FP64;
    char* W = wsb(ctx);
    double* diag = reinterpret_cast<double*>(W + p.off_diag);
    double* gram = reinterpret_cast<double*>(W + p.off_gram);
    FO_CUDA(launch_diag_sums(S.t, (int64_t)p.slot_bytes, p.n_tslots, p.n, p.np, is64, diag, st), "diag_sums");
    if (p.m > 1 && p.k > 1)
        FO_CUDA(launch_gram(S.t, (int64_t)p.slot_bytes, p.k - 1, p.m - 1, 0, p.k - 1, p.np, is64,
                            reinterpret_cast<double*>(W + p.off_gpart), p.gram_nblocks, gram, st),
                "gram");
    FO_CUDA(launch_assemble_moments(diag, gram, p.k, p.m, p.n_terms, p.n,
                                    reinterpret_cast<double*>(W + p.off_tau), st),
            "moments");
    return FO_OK;
}

// Coefficients at the device mu and their conversion to giant-step coefficients g.
fo_status coefficients(fo_ctx* ctx, const Plan& p, double kT, cudaStream_t st, int* launches) {
    char* W = wsb(ctx);
    double* ct = reinterpret_cast<double*>(W + p.off_ct);
    double* f = reinterpret_cast<double*>(W + p.off_f);
    double* c = reinterpret_cast<double*>(W + p.off_c);
    double* g = reinterpret_cast<double*>(W + p.off_g);
    FO_CUDA(launch_fermi_nodes(p.M, ct, ctx->res, kT, f, st), "fermi_nodes");
    FO_CUDA(launch_coeffs(f, ct, p.M, p.n_terms, p.km, c, st), "coeffs");
    FO_CUDA(launch_g_convert(c, p.k, p.m, g, st), "g_convert");
    *launches += 3;
    if (p.moments) {
        FO_CUDA(launch_poly_trace(c, reinterpret_cast<double*>(W + p.off_tau), p.n_terms, ctx->res, st),
                "poly_trace");
        *launches += 1;
    }
    return FO_OK;
}

// R_l = sum_i g_{i,l} T_i for every l (the S_j sums of the paper in the Chebyshev basis).
fo_status contraction(fo_ctx* ctx, const Plan& p, const Slots& S, double* dP, int64_t ldp,
                      cudaStream_t st, int* launches) {
    const double* g = reinterpret_cast<const double*>(wsb(ctx) + p.off_g);
    if (p.prec == FO_PREC_FP64) {
        FO_CUDA(launch_contract_f64(g, p.k, p.m, S.Td(0), (int64_t)(p.slot_bytes / 8), S.Rd(0),
                                    (int64_t)(p.slot_bytes / 8), p.n, p.np, st),
                "contract");
    } else {
        FO_CUDA(launch_contract_f32(g, p.k, p.m, S.T(0).x, (int64_t)(p.slot_bytes / 4), S.R(0).x,
                                    (int64_t)(p.slot_bytes / 4), p.n, p.np, p.m > 1 ? p.planes : 0,
                                    p.fp16, p.pscale_r, p.np * p.np, st, ctx->flag + 1),
                "contract");
    }
    *launches += 1;
    if (p.m == 1) {
        if (p.prec == FO_PREC_FP64)
            FO_CUDA(launch_copy_out(S.Rd(0), p.np, p.n, dP, ldp, st), "copy_out");
        else
            FO_CUDA(launch_copy_out_f32(S.R(0).x, p.np, p.n, dP, ldp, st), "copy_out");
        *launches += 1;
    }
    return FO_OK;
}

// Clenshaw recurrence in Y = T_k: b_{m-1} = R_{m-1}; b_l = 2 Y b_{l+1} - b_{l+2} + R_l;
// P = Y b_1 - b_2 + R_0 (written as float64 into dP). b_l overwrites R_l in place.
fo_status clenshaw(fo_ctx* ctx, const Plan& p, const Slots& S, double* dP, int64_t ldp,
                   cudaStream_t st, int sym, int* n_gemm) {
    if (p.m == 1) return FO_OK;
    const int ysl = giant_slot(p, 1);
    for (int l = p.m - 2; l >= 1; --l) {
        Product q;
        q.a = ysl;
        q.b = l + 1; q.b_r = true;
        q.d = l; q.d_r = true;
        q.out = l; q.out_r = true;
        q.alpha = 2.0;
        q.tag = "clenshaw";
        q.index = l;
        if (l + 2 <= p.m - 1) { q.c = l + 2; q.c_r = true; q.beta = -1.0; }
        FO_TRY(run_product(ctx, p, S, q, st, sym));
        ++*n_gemm;
    }
    Product q;
    q.a = ysl;
    q.b = 1; q.b_r = true;
    q.d = 0; q.d_r = true;
    q.alpha = 1.0;
    if (p.m >= 3) { q.c = 2; q.c_r = true; q.beta = -1.0; }
    q.out64 = dP;
    q.ldo = ldp;
    q.tag = "final";
    FO_TRY(run_product(ctx, p, S, q, st, sym));
    ++*n_gemm;
    return FO_OK;
}

fo_status check_params(fo_ctx* ctx, const fo_params* prm) {
    if (!prm) return fail(ctx, FO_ERR_ARG, "params is NULL");
    if (!(prm->kT > 0.0) || !std::isfinite(prm->kT)) return fail(ctx, FO_ERR_ARG, "kT must be > 0");
    if (prm->use_given_bounds && !(prm->emax > prm->emin))
        return fail(ctx, FO_ERR_ARG, "emax must exceed emin");
    if (prm->mu_mode < FO_MU_FIXED || prm->mu_mode > FO_MU_LEARNED)
        return fail(ctx, FO_ERR_ARG, "unknown mu_mode");
    if (prm->mu_mode == FO_MU_LEARNED) return fail(ctx, FO_ERR_UNSUPPORTED, "learned mu needs a trained model");
    return FO_OK;
}

fo_status density_impl(fo_ctx* ctx, const double* dH, int64_t n, int64_t ld, double n_e,
                       const fo_params* prm, double* dP, int64_t ldp, fo_result* res,
                       cudaStream_t st) {
    FO_TRY(check_params(ctx, prm));
    if (!dH || !dP) return fail(ctx, FO_ERR_ARG, "H and P must be non-NULL");
    if (ld < n || ldp < n) return fail(ctx, FO_ERR_ARG, "leading dimensions must be >= n");
    const bool bisect = prm->mu_mode == FO_MU_BISECT;
    if (bisect && !(n_e >= 0.0 && n_e <= (double)n)) return fail(ctx, FO_ERR_ARG, "n_e must be in [0, n]");
    Plan p;
    FO_TRY(make_plan(ctx, n, prm->n_terms, prm->k, prm->precision, bisect, bisect, prm->n_quad, &p));
    FO_TRY(ensure_ws(ctx, p.total));
    Slots S{wsb(ctx) + p.off_t, wsb(ctx) + p.off_r, p.slot_bytes, p.np, p.planes};
    const int sym = 1;  // symmetric products (upper-triangle tiles, mirrored)
    int n_gemm = 0, launches = 0, lstage = 0;
    char* W = wsb(ctx);
    double* part = reinterpret_cast<double*>(W + p.off_part);
    const int hcall = prof_begin(ctx, st, FO_STAGE_CALL);

    // spectral bounds and X = scaled H (split into planes for the tensor-core forms)
    int h = prof_begin(ctx, st, FO_STAGE_BOUNDS);
    FO_CUDA(cudaMemsetAsync(ctx->res, 0, sizeof(DevResult), st), "memset");
    FO_CUDA(launch_gershgorin(dH, n, ld, part, part + p.nparts, reinterpret_cast<int*>(part + 2 * p.nparts),
                              p.nparts, ctx->res, prm->use_given_bounds, prm->emin, prm->emax, st),
            "bounds");
    FO_TRY(pack_x(ctx, p, S, dH, ld, st));
    lstage = (prm->use_given_bounds ? 1 : 2) + 1;
    prof_end(ctx, st, h, 0.0, lstage);
    launches += lstage;

    // baby steps T_2 .. T_k
    const int g0 = n_gemm;
    FO_TRY(baby_steps(ctx, p, S, p.k, st, sym, &n_gemm));
    double* ct = reinterpret_cast<double*>(W + p.off_ct);
    FO_CUDA(launch_cos_table(p.M, ct, st), "cos_table");
    launches += 1;
    const int max_it = prm->max_bisect > 0 ? prm->max_bisect : 200;
    if (bisect) {
        // giant steps T_{2k} .. T_{(m-1)k}, exact moments, bisection for mu
        if (p.giants) FO_TRY(giant_steps(ctx, p, S, st, sym, &n_gemm));
        h = prof_begin(ctx, st, FO_STAGE_MOMENTS);
        FO_TRY(exact_moments(ctx, p, S, st));
        lstage = 1 + ((p.m > 1 && p.k > 1) ? 2 : 0) + 1;
        prof_end(ctx, st, h, 0.0, lstage);
        launches += lstage;
        h = prof_begin(ctx, st, FO_STAGE_MU);
        double* w = reinterpret_cast<double*>(W + p.off_w);
        FO_CUDA(launch_dos_weights(reinterpret_cast<double*>(W + p.off_tau), p.n_terms, p.M, ct, w, st),
                "dos_weights");
        FO_CUDA(launch_bisect(w, ct, p.M, ctx->res, prm->kT, n_e, max_it, st), "bisect");
        prof_end(ctx, st, h, 0.0, 2);
        launches += 2;
    } else {
        // fixed mu: write it into the device record (kept after the bounds pass)
        FO_CUDA(launch_set_scalar(&ctx->res->mu, prm->mu, st), "mu");
        launches += 1;
    }
    h = prof_begin(ctx, st, FO_STAGE_COEFFS);
    lstage = 0;
    FO_TRY(coefficients(ctx, p, prm->kT, st, &lstage));
    prof_end(ctx, st, h, 0.0, lstage);
    launches += lstage;
    h = prof_begin(ctx, st, FO_STAGE_CONTRACT);
    lstage = 0;
    FO_TRY(contraction(ctx, p, S, dP, ldp, st, &lstage));
    prof_end(ctx, st, h, 0.0, lstage);
    launches += lstage;
    FO_TRY(clenshaw(ctx, p, S, dP, ldp, st, sym, &n_gemm));
    launches += n_gemm - g0;
    h = prof_begin(ctx, st, FO_STAGE_TRACE);
    FO_CUDA(launch_trace_frob(dP, n, ldp, part, p.nparts, ctx->res, st), "trace");
    prof_end(ctx, st, h, 0.0, 2);
    launches += 2;
    prof_end(ctx, st, hcall, product_flops(p) * n_gemm, launches);
    if (ctx->prof) ctx->prof_calls += 1;

    if (res && !(prm->flags & FO_FLAG_NO_RESULT_SYNC)) {
        DevResult hr;
        int flag[5] = {0, 0, 0, 0, 0};
        FO_CUDA(cudaMemcpyAsync(&hr, ctx->res, sizeof(DevResult), cudaMemcpyDeviceToHost, st), "readback");
        FO_CUDA(cudaMemcpyAsync(flag, ctx->flag, sizeof(flag), cudaMemcpyDeviceToHost, st), "readback");
        FO_CUDA(cudaStreamSynchronize(st), "sync");
        if (flag[1] != 0)
            return fail(ctx, FO_ERR_CUDA, "self-check violation code " + std::to_string(flag[1]) + " (" +
                                              std::to_string(flag[2]) + ", " + std::to_string(flag[3]) + ")");
        std::memset(res, 0, sizeof(*res));
        res->mu = hr.mu;
        res->trace = hr.trace;
        res->trace_poly = hr.trace_poly;
        res->frob2 = hr.frob2;
        res->emin = hr.bounds[0];
        res->emax = hr.bounds[1];
        res->k = p.k;
        res->m = p.m;
        res->n_gemm = n_gemm;
        res->bisect_iters = hr.iters;
        res->learned_accepted = 0;
        res->n_launches = launches;
        int status = hr.status;
        if (flag[0]) status = FO_ERR_DEVICE_TIMEOUT;
        res->status = status;
        if (status != FO_OK)
            return fail(ctx, (fo_status)status, std::string("device stage failed: ") +
                                                    fo_status_string((fo_status)status));
    }
    return FO_OK;
}

}  // namespace

extern "C" {

const char* fo_version(void) { return "fermi-gb300 0.1"; }

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
    if (cudaMalloc(&ctx->res, sizeof(DevResult)) != cudaSuccess ||
        cudaMalloc(&ctx->flag, 8 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->res) cudaFree(ctx->res);
        delete ctx;
        return FO_ERR_NOMEM;
    }
    cudaMemset(ctx->res, 0, sizeof(DevResult));
    cudaMemset(ctx->flag, 0, 8 * sizeof(int));
    *out = ctx;
    return FO_OK;
}

fo_status fo_destroy(fo_ctx* ctx) {
    if (!ctx) return FO_OK;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        prof_collect(ctx);
        for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
        if (ctx->ws) cudaFree(ctx->ws);
        if (ctx->stage) cudaFree(ctx->stage);
        if (ctx->res) cudaFree(ctx->res);
        if (ctx->flag) cudaFree(ctx->flag);
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
    const int nparts = 2 * ctx->num_sms;
    FO_TRY(ensure_ws(ctx, align256(8 * 3 * (size_t)nparts + 64)));
    double* part = reinterpret_cast<double*>(ctx->ws);
    FO_CUDA(launch_gershgorin(dH, n, ld, part, part + nparts, reinterpret_cast<int*>(part + 2 * nparts),
                              nparts, ctx->res, 0, 0.0, 0.0, st),
            "bounds");
    FO_CUDA(launch_export_bounds(ctx->res, d_bounds, st), "bounds export");
    return FO_OK;
}

fo_status fo_chebyshev_coeffs(fo_ctx* ctx, double kT, double mu, double emin, double emax,
                              int32_t n_terms, int32_t n_quad, double* d_c, void* stream) {
    if (!ctx) return FO_ERR_ARG;
    if (!d_c || n_terms < 1 || n_terms > 4096) return fail(ctx, FO_ERR_ARG, "bad n_terms or output");
    if (!(kT > 0.0) || !(emax > emin)) return fail(ctx, FO_ERR_ARG, "need kT > 0 and emax > emin");
    DeviceGuard g(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int M = n_quad > 0 ? n_quad : (2048 > 4 * n_terms ? 2048 : 4 * n_terms);
    if (M < n_terms) return fail(ctx, FO_ERR_ARG, "n_quad must be >= n_terms");
    const size_t need = align256(8 * 4 * (size_t)M) + align256(8 * (size_t)M);
    FO_TRY(ensure_ws(ctx, need));
    double* ct = reinterpret_cast<double*>(ctx->ws);
    double* f = reinterpret_cast<double*>(wsb(ctx) + align256(8 * 4 * (size_t)M));
    FO_CUDA(launch_set_bounds(ctx->res, emin, emax, st), "set_bounds");
    FO_CUDA(launch_set_scalar(&ctx->res->mu, mu, st), "mu");
    FO_CUDA(launch_cos_table(M, ct, st), "cos_table");
    FO_CUDA(launch_fermi_nodes(M, ct, ctx->res, kT, f, st), "fermi_nodes");
    FO_CUDA(launch_coeffs(f, ct, M, n_terms, n_terms, d_c, st), "coeffs");
    return FO_OK;
}

fo_status fo_density_matrix(fo_ctx* ctx, const double* dH, int64_t n, int64_t ld, double n_e,
                            const fo_params* params, double* dP, int64_t ldp, fo_result* res,
                            void* stream) {
    if (!ctx) return FO_ERR_ARG;
    DeviceGuard g(ctx->device);
    return density_impl(ctx, dH, n, ld, n_e, params, dP, ldp, res, reinterpret_cast<cudaStream_t>(stream));
}

fo_status fo_density_matrix_host(fo_ctx* ctx, const double* hH, int64_t n, int64_t ld, double n_e,
                                 const fo_params* params, double* hP, int64_t ldp, fo_result* res,
                                 void* stream) {
    if (!ctx) return FO_ERR_ARG;
    if (!hH || !hP || n < 1 || ld < n || ldp < n) return fail(ctx, FO_ERR_ARG, "bad arguments");
    DeviceGuard g(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t mat = align256((size_t)n * n * 8);
    if (ctx->stage_bytes < 2 * mat) {
        if (ctx->stage) {
            cudaDeviceSynchronize();
            cudaFree(ctx->stage);
            ctx->stage = nullptr;
            ctx->stage_bytes = 0;
        }
        if (cudaMalloc(&ctx->stage, 2 * mat) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, FO_ERR_NOMEM, "staging allocation failed");
        }
        ctx->stage_bytes = 2 * mat;
    }
    double* dH = reinterpret_cast<double*>(ctx->stage);
    double* dP = reinterpret_cast<double*>(reinterpret_cast<char*>(ctx->stage) + mat);
    FO_CUDA(cudaMemcpy2DAsync(dH, n * 8, hH, ld * 8, n * 8, n, cudaMemcpyHostToDevice, st), "H2D");
    fo_params prm = *params;
    prm.flags &= ~FO_FLAG_NO_RESULT_SYNC;
    fo_result local;
    fo_status s = density_impl(ctx, dH, n, n, n_e, &prm, dP, n, res ? res : &local, st);
    if (s != FO_OK && s != FO_ERR_NOT_CONVERGED) return s;
    FO_CUDA(cudaMemcpy2DAsync(hP, ldp * 8, dP, n * 8, n * 8, n, cudaMemcpyDeviceToHost, st), "D2H");
    FO_CUDA(cudaStreamSynchronize(st), "sync");
    return s;
}

fo_status fo_moments(fo_ctx* ctx, const double* dH, int64_t n, int64_t ld, const double* d_bounds,
                     int32_t n_moments, int32_t precision, double* d_tau, void* stream) {
    if (!ctx) return FO_ERR_ARG;
    if (!dH || !d_bounds || !d_tau || n < 1 || ld < n || n_moments < 1 || n_moments > 256)
        return fail(ctx, FO_ERR_ARG, "bad arguments");
    DeviceGuard g(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int K = n_moments <= 2 ? 1 : (n_moments + 1) / 2;
    Plan p;
    // k = K baby steps, m = 2: the assembly then covers tau_0 .. tau_{2K-1}
    FO_TRY(make_plan(ctx, n, 2 * K, K, precision, false, true, 0, &p));
    FO_TRY(ensure_ws(ctx, p.total));
    Slots S{wsb(ctx) + p.off_t, wsb(ctx) + p.off_r, p.slot_bytes, p.np, p.planes};
    const int sym = 1;  // symmetric products (upper-triangle tiles, mirrored)
    FO_CUDA(cudaMemcpyAsync(ctx->res->bounds, d_bounds, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st),
            "bounds");
    FO_TRY(pack_x(ctx, p, S, dH, ld, st));
    int n_gemm = 0;
    FO_TRY(baby_steps(ctx, p, S, p.k, st, sym, &n_gemm));
    FO_TRY(exact_moments(ctx, p, S, st));
    FO_CUDA(cudaMemcpyAsync(d_tau, wsb(ctx) + p.off_tau, 8 * (size_t)n_moments, cudaMemcpyDeviceToDevice, st),
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
    Plan p;
    FO_TRY(make_plan(ctx, n, 4, 2, precision, false, false, 0, &p));
    // slots: 0 = A, 1 = B, 2 = C, 3 = D, 4 = out
    const size_t bytes = p.slot_bytes * 5;
    FO_TRY(ensure_ws(ctx, bytes));
    Slots S{wsb(ctx), wsb(ctx), p.slot_bytes, p.np, p.planes};
    const float ps = p.fp16 ? p.pscale_t : 1.0f;
    FO_CUDA(launch_pack_f32(dA, n, ld, S.T(0), p.np, p.planes, p.fp16, ps, st), "pack");
    FO_CUDA(launch_pack_f32(dB, n, ld, S.T(1), p.np, p.planes, p.fp16, ps, st), "pack");
    if (dC) FO_CUDA(launch_pack_f32(dC, n, ld, S.T(2), p.np, 0, 0, 1.0f, st), "pack");
    if (dD) FO_CUDA(launch_pack_f32(dD, n, ld, S.T(3), p.np, 0, 0, 1.0f, st), "pack");
    Epilogue ep;
    std::memset(&ep, 0, sizeof(ep));
    ep.alpha = (float)((double)alpha / ((double)ps * ps));
    ep.beta = beta;
    ep.shift = shift;
    ep.n_real = (int32_t)n;
    ep.C = dC ? S.T(2).x : nullptr;
    ep.D = dD ? S.T(3).x : nullptr;
    ep.ld = p.np;
    ep.out = S.T(4);
    ep.planes = 0;
    ep.fp16 = p.fp16;
    ep.plane_scale = 1.0f;
    ep.dbg = ctx->flag + 1;
    std::string err;
    cudaError_t e = tc_gemm(p.prec, p.np, S.T(0), S.T(1), ep, symmetric ? 1 : 0, ctx->flag, st, &err);
    if (e != cudaSuccess) return err.empty() ? cuda_fail(ctx, e, "tc_gemm") : fail(ctx, FO_ERR_CUDA, err);
    FO_CUDA(cudaMemcpy2DAsync(dOut, ld * 4, S.T(4).x, p.np * 4, n * 4, n, cudaMemcpyDeviceToDevice, st),
            "copy out");
    return FO_OK;
}

}  // extern "C"
