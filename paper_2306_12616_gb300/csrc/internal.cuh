// Internal declarations shared by the CUDA translation units of the solver.
//
// Every call runs on a batch plan: one or more independent Hamiltonians ("instances"),
// each with its own size, sharing the expansion parameters (number of terms, k, m,
// arithmetic). Each stage of the method is one launch over the whole batch: a kernel
// finds its instance either from blockIdx.y (stages with the same work per instance) or
// from a per-instance prefix sum of block counts (stages whose work grows with the
// instance size: the block-to-instance map is a binary search on the prefix).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "fermi.h"

namespace fo {

// Every working matrix is stored n_pad x n_pad (row-major, leading dimension n_pad) with a
// zero border, n_pad a multiple of kPad; the tensor-core tiles then never straddle an edge
// and the zero border stays zero through every polynomial step because the identity is
// only ever applied to the first n rows (the algebra of X restricted to the n-dim block).
constexpr int kPad = 128;

// Device-resident record of the scalar results of one instance.
struct DevResult {
    double bounds[2];     // emin, emax
    double mu;
    double trace;         // tr P
    double frob2;         // ||P||_F^2
    double trace_poly;    // sum_n c_n tau_n at mu
    int32_t iters;        // mu search evaluations
    int32_t status;       // fo_status of device stages
    int32_t nonfinite;    // H held NaN/Inf
    int32_t learned_ok;   // learned mu accepted
    int32_t active;       // 0: every kernel skips this instance
    int32_t evals;        // evaluations of P (learned mode)
    int32_t fixed;        // the trace correction was applied
    int32_t m_eff;        // giant-step count of this instance's expansion (learned order); 0: the plan's m
    int32_t n_eff;        // coefficients of this instance's expansion (learned order); 0: the plan's
    double mu_lo, mu_hi;  // final bracket of the mu search
    double mu0;           // learned proposal (learned mode)
    double mu_prev, tr_prev;  // previous evaluation (learned mode secant)
    double order;         // learned expansion order (learned mode)
    double kt_eff;        // effective temperature of the truncated expansion (learned mode)
    double trace_raw;     // tr P as the expansion produced it, before the trace correction
    double gamma;         // trace correction P += gamma (P - P^2) (0 unless fixed)
    double proj;          // residual removed by the trace projection, per diagonal entry
};

// Per-instance descriptor, written once per plan. slots: the instance's slot region,
// T slots (baby steps, then giant steps) followed by the R / Clenshaw slots; a slot holds
// a float64 matrix, or a float32 master followed by its 16-bit planes (plane p at byte
// 4 np^2 + 2 p np^2 of the slot).
struct Inst {
    int64_t n, np;
    char* slots;
    int64_t slot_bytes;
    double* c;            // km coefficients
    double* g;            // k x m giant-step coefficients, l-major
    double* tau;          // km + 2 moments
    double* w;            // M DOS weights
    double* f;            // M Fermi values at the nodes
    double* diag;         // traces of the T slots
    double* gram;         // Frobenius products, giant-major
    double* gpart;        // gram partials, gram_blocks x npairs
    DevResult* res;
    double* lz;           // Lanczos state: 3 np + 2 kLzMax + 3 doubles
    int32_t bucket;       // tensor-map bucket (instances of equal np)
    int32_t in_bucket;    // index within the bucket
    int32_t gram_blocks;  // blocks of the Frobenius-product kernel for this instance
    int32_t user;         // index of the instance in the caller's arrays
};

// Per-call inputs of an instance (written at the start of every call).
struct InstIO {
    const double* H;
    double* P;
    int64_t ldh, ldp;
    double kT, n_e, mu;       // mu: FO_MU_FIXED value
    double emin, emax;        // given bounds
    const double* bounds_src; // device bounds to copy (fo_moments), or null
};

// Plan-wide constants.
struct Shape {
    int32_t k, m, km, n_terms, M;
    int32_t n_tslots;     // T slots per instance (R slot l is n_tslots + l)
    int32_t planes, fp16, is64;
    int32_t ublk;         // 1: the slots' 16-bit planes hold the 128-blocks on and above the
                          // diagonal only (a lower block is read transposed by the products)
    float pscale_t, pscale_r;
};

// One recurrence product of the whole batch (slot indices are per instance):
//   out = alpha * A B^T + beta * C + D + shift * I_n
struct Step {
    int32_t a, b, c, d, out;   // -1 = absent
    int32_t out64;             // 1: write the instance's float64 P (InstIO) instead of a slot
    int32_t planes;            // 16-bit planes to write for out
    int32_t fp16;
    int32_t lower_master;      // symmetric mode: also write the float32 master below the
                               // diagonal (the solver's slots keep it above the diagonal only)
    int32_t need_m;            // instances whose expansion stops at m_eff <= need_m giant steps
                               // skip this product (its output is zero or unused for them)
    int32_t fix64;             // with out64: P <- P + gamma (P - alpha A B^T) in float64, P the
                               // instance's float64 P (read and rewritten), gamma = res->gamma
    float alpha, beta, shift;  // float32 path; alpha includes the fp16 plane scales
    float plane_scale;
    double alpha64, beta64, shift64;
    double* part;              // with out64: (tr, ||.||_F^2) partials of the float64 result per
                               // 128 x 128 block on and above the diagonal, 2 doubles per block
    const int* part_pre;       // block prefix per instance (the 128-wide tile work list)
    int* dbg;                  // self-check record (null unless built with FO_SELF_CHECK)
};

// Up to kMaxSteps independent products of the whole batch in one launch (a stage of the
// staged recurrences): CTA b computes step b / tiles, tile b % tiles of the step.
constexpr int kMaxSteps = 16;
struct StepList {
    Step s[kMaxSteps];
    int32_t count;
};

// A chain of dependent products of the whole batch in one launch (the baby steps, the giant
// steps or the Clenshaw recurrence: step s reads what step s - 1 wrote). Every CTA takes a
// ticket from `ticket` when it starts; tickets run window by window (consecutive instances),
// within a window step by step, within a step tile by tile, so a tile's dependencies always
// hold smaller tickets, taken by CTAs that are already running. A tile of step s waits until
// `done[instance]` counts s x (tiles per step of that instance), and adds one when its stores
// are complete. Both counters are zeroed before the launch.
constexpr int kMaxChain = 128;
constexpr int kMaxWin = 64;
struct ChainList {
    Step s[kMaxChain];
    int32_t count;                 // steps
    int32_t nwin;                  // windows
    int32_t win_base[kMaxWin + 1]; // first ticket of window w; win_base[nwin] = all tickets
    int32_t win_i0[kMaxWin + 1];   // first instance of window w; win_i0[nwin] = end instance
    int* ticket;
    int* done;
    int32_t drop;                  // a ticket whose tile does not signal (timeout tests); -1: none
};

// The block-to-instance map of a grouped launch: pre[j] = blocks of instances < j.
struct Work {
    const int* pre;   // device, count + 1 entries
    int count;        // instances
    int total;        // blocks
};

// Whether a product step is computed for an instance: it is active, and its expansion (cut at
// m_eff giant steps by a learned order) needs the step's output.
__device__ __forceinline__ bool step_needed(const DevResult* r, int need_m) {
    return r->active && !(r->m_eff > 0 && r->m_eff <= need_m);
}
// Number of coefficients of an instance's expansion (the plan's unless a learned order cut it).
__device__ __forceinline__ int eff_terms(const DevResult* r, int n_terms) {
    return r->n_eff > 0 ? r->n_eff : n_terms;
}

// Largest j in [lo, hi) with pre[j] <= b (pre ascending, pre[lo] <= b < pre[hi]).
__device__ __forceinline__ int find_inst(const int* __restrict__ pre, int lo, int hi, int b) {
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pre + mid) <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Tile (bi, bj), bj >= bi, that is the b-th of the upper triangle of a tn x tn tile grid in
// row-major order: row bi holds tn - bi tiles, so the rows before it hold
// P(bi) = bi tn - bi (bi - 1) / 2. bi is the root of P(x) = b, estimated by a float32 square
// root and corrected exactly (a loop over the rows would cost O(tn) per block).
__device__ __forceinline__ void upper_tile(int b, int tn, int& bi, int& bj) {
    const float e = 2.0f * (float)tn + 1.0f;
    const float d = e * e - 8.0f * (float)b;
    int r = (int)((e - sqrtf(d > 0.0f ? d : 0.0f)) * 0.5f);
    if (r < 0) r = 0;
    if (r > tn - 1) r = tn - 1;
    auto P = [&](int x) { return x * tn - x * (x - 1) / 2; };
    while (r > 0 && P(r) > b) --r;
    while (r + 1 < tn && P(r + 1) <= b) ++r;
    bi = r;
    bj = r + (b - P(r));
}

// Asynchronous 16-byte global -> shared copies (cp.async, L2 only) and their group waits.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ------------------------------------------------- mbarriers and bounded waits
// Every wait on the device is bounded: a legitimate wait is microseconds; on expiry the
// kernel raises the device error flag, drains what it has in flight and returns.
constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s: a legitimate wait is microseconds
constexpr uint64_t kDrainNs = 200000000ull;   // 0.2 s for draining after an abort

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait. Returns false when the deadline passes or another role aborted.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns,
                                 volatile int* abort_flag) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u) {
            if (abort_flag && *abort_flag) return false;
            const uint64_t t = gtimer();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) return false;
        }
    }
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Warp-uniform bounded wait: every lane observes the phase; the exit decision is shared.
__device__ inline bool mbar_wait_warp(uint64_t* bar, uint32_t parity, uint64_t limit_ns,
                                      volatile int* abort_flag) {
    const int lane = threadIdx.x & 31;
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        const bool done = mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, done)) return true;
        if ((it & 255u) == 255u) {
            int stop = 0;
            if (lane == 0) {
                if (abort_flag && *abort_flag) stop = 1;
                const uint64_t t = gtimer();
                if (t0 == 0) t0 = t;
                else if (t - t0 > limit_ns) stop = 1;
            }
            if (__shfl_sync(0xffffffffu, stop, 0)) return false;
        }
    }
}


// Packed float32 FMA: __ffma2_rn (sm_100 and later) forms a * b + c on both halves of a float2
// at once, the same round-to-nearest result per half as fmaf at half the instruction count.
// The builtin keeps the operands in register pairs the compiler allocates itself (inline
// PTX on 64-bit integers cost a register move per FMA).

// Elementwise row blocks: a block covers ew_rows(np) rows (about 8192 entries).
__host__ __device__ inline int ew_rows(int64_t np) {
    const int64_t r = 8192 / np;
    return r < 1 ? 1 : (int)r;
}
__host__ __device__ inline int ew_blocks(int64_t np) {
    const int r = ew_rows(np);
    return (int)((np + r - 1) / r);
}
// Contraction of the float32 forms: the upper triangle is walked as 16-byte quads (row r
// holds the quads from column 4 floor(r / 4) to np - 4), ct_threads(k) thread pairs per block,
// one quad per pair and step (each thread of the pair stages half of the k - 1 quads and forms
// half of the R_l), kCtSteps steps per block.
constexpr int kCtSteps = 16;
__host__ __device__ inline int ct_threads(int) {
    // 64 pairs: the two ring stages take 2 (k - 1) 1 KB (39 KB at k = 20, 126 KB at the largest
    // k = 64), so that up to four blocks share an SM (128 registers per thread); small blocks
    // measured faster than 128 or 256 pairs, and deeper rings than two stages slower
    return 64;
}
__host__ __device__ inline int64_t ct_quads(int64_t np) { return np * (np + 4) / 8; }
__host__ __device__ inline int ct_blocks(int64_t np, int k) {
    const int64_t per = (int64_t)ct_threads(k) * kCtSteps;
    return (int)((ct_quads(np) + per - 1) / per);
}
// Reduction row blocks (traces of P): about 16K entries per block, so that the loads of a
// float64 P are spread over enough blocks to be in flight together.
__host__ __device__ inline int red_rows(int64_t np) {
    const int64_t r = 16384 / np;
    return r < 1 ? 1 : (int)r;
}
__host__ __device__ inline int red_blocks(int64_t np) {
    const int r = red_rows(np);
    return (int)((np + r - 1) / r);
}
constexpr int kGershRows = 8;   // rows per block of the bounds kernel (a warp per row)
constexpr int kLzMax = 64;      // Lanczos steps at most

// Self-check build (-DFO_SELF_CHECK): kernels verify the index range and the alignment of
// their global accesses, record the first violation in dbg[0..3] and skip the access.
#ifdef FO_SELF_CHECK
#define FO_CHK(dbg, cond, code, v1, v2)                                           \
    ((cond) ? true                                                               \
            : ((dbg) ? (atomicCAS((int*)(dbg), 0, (code)) == 0                   \
                            ? ((dbg)[1] = (int)(v1), (dbg)[2] = (int)(v2), false) \
                            : false)                                             \
                     : false))
#else
#define FO_CHK(dbg, cond, code, v1, v2) true
#endif

// ---------------------------------------------------------------- reduce.cu
// Resets every instance's DevResult and writes its per-call inputs (ios[0..count)).
cudaError_t launch_set_io(const InstIO* ios, int count, InstIO* d_io, const Inst* d_inst, int first,
                          cudaStream_t s);
// Gershgorin bounds (use_given = 0) or the given / copied bounds (use_given = 1).
cudaError_t launch_bounds(const Inst* in, const InstIO* io, int batch, Work wg, double* part,
                          int use_given, cudaStream_t s);
// Lanczos bounds (after the Gershgorin bounds): `steps` float64 Lanczos steps on H, extreme
// Ritz values widened by their residuals and 1% of the width, clamped to Gershgorin.
cudaError_t launch_lanczos(const Inst* in, const InstIO* io, int batch, Work wg, double* part, int steps,
                           cudaStream_t s, int* launches);
// d_bounds[0..2] = emin, emax, non-finite flag of one instance.
cudaError_t launch_export_bounds(const DevResult* res, double* out3, cudaStream_t s);
// X = (2H - (emin+emax) I)/(emax - emin) into slot 0 of every instance.
cudaError_t launch_scale(const Inst* in, const InstIO* io, Work ws, const Shape& sh, cudaStream_t s,
                         int* dbg);
cudaError_t launch_diag_sums(const Inst* in, int batch, int count, const Shape& sh, cudaStream_t s);
// gram[(g0 + g) * nbaby + b] = <slot giant0 + g, slot baby0 + b> for every instance.
// Geometry of the float32 masters for the tensor maps of the Frobenius-product kernel: per
// bucket of equally sized instances the master of slot 0 of its first instance, the strides
// of slots and instances; per launch group (at most kMaxBuckets buckets) its instances.
struct GramBucket {
    const char* master0;
    int64_t np, slot_bytes, inst_bytes;
    int count;
};
struct GramGroup {
    int b0, nb, i0, i1;   // buckets [b0, b0 + nb) hold instances [i0, i1)
};
struct GramGeom {
    const GramBucket* bk;
    const GramGroup* grp;
    int ngroups;
    int nslots;           // slots per instance
    const int* pre_host;  // host copy of the Frobenius kernel's unit prefix (Work::pre)
};
// 4-D tensor map (column, row, slot, instance) over a bucket's float32 masters, box of 128
// columns x 1 row x box_slots slots x 1 instance, no swizzle.
bool gram_make_map(void* map128, const GramBucket& b, int nslots, int box_slots, std::string* err);
// geom: the tensor-map geometry of float32 masters (null: the cp.async kernel, as for float64)
cudaError_t launch_gram(const Inst* in, int batch, Work wgr, int giant0, int ngiant, int baby0,
                        int nbaby, int out_g0, int is64, const GramGeom* geom, int* err, cudaStream_t s,
                        int* launches);
// tau_0 .. tau_{n_terms-1} from the traces and the Frobenius products.
cudaError_t launch_assemble_moments(const Inst* in, int batch, const Shape& sh, cudaStream_t s);
cudaError_t launch_trace_frob(const Inst* in, const InstIO* io, Work wr, double* part, cudaStream_t s);
// tr P and ||P||_F^2 of every instance from the per-block partials of its float64-output
// product (prefix `pre` of the 128 x 128 blocks on and above the diagonal, batch + 1 entries). mode 0: the result's trace; mode 1: the
// trace before the correction and the correction's gamma = (N_e - tr P)/(tr P - ||P||_F^2)
// (every instance without a failed stage is made active again); mode 2: the trace after the
// correction, whose float64 residual is then removed by the trace projection of P's diagonal.
cudaError_t launch_tile_trace(const Inst* in, const InstIO* io, int batch, const int* pre, const double* part,
                              int mode, cudaStream_t s);
cudaError_t launch_copy_out(const Inst* in, const InstIO* io, Work we, const Shape& sh, cudaStream_t s);
// Standalone packing of a float32 matrix into slot `slot` (fo_recurrence_product).
cudaError_t launch_pack_f32(const float* A, int64_t n, int64_t lda, char* slot, int64_t np, int planes,
                            int fp16, float pscale, cudaStream_t s);
// Blocks of the Frobenius-product kernel for one instance (upper-triangle chunks).
int gram_blocks_for(int64_t np, int is64);

// ------------------------------------------------------------------- mlp.cu
// Learned chemical potential: 68 inputs (64 moments, N_e/N, kT_x, e_a/100, e_b/100),
// two hidden layers of 256 SiLU units, 2 outputs (mu_x, order), float32 parameters stored
// W1 (256 x 68), b1, W2 (256 x 256), b2, W3 (2 x 256), b3; normalisation vector
// [feature mean (68), feature std (68), target mean (2), target std (2)].
constexpr int kMlpMoments = 64;
constexpr int kMlpIn = kMlpMoments + 4;
constexpr int kMlpHidden = 256;
constexpr int kMlpOut = 2;
constexpr int kMlpNorm = 2 * kMlpIn + 2 * kMlpOut;
constexpr float kMlpLossW0 = 1.0f;   // weight of the mu_x error
constexpr float kMlpLossW1 = 0.1f;   // weight of the order error
// The order target: the smallest L with sum_{j >= L} |c_j| <= kOrderEps. |T_j| <= 1 on the
// scaled spectrum, so the expansion cut there is within kOrderEps of the full one in the
// 2-norm (a quarter of the split forms' 1e-6 bar).
constexpr double kOrderEps = 2.5e-7;
struct MlpOffsets {
    int W1, b1, W2, b2, W3, b3, total;
};
inline MlpOffsets mlp_offsets() {
    MlpOffsets o;
    o.W1 = 0;
    o.b1 = o.W1 + kMlpHidden * kMlpIn;
    o.W2 = o.b1 + kMlpHidden;
    o.b2 = o.W2 + kMlpHidden * kMlpHidden;
    o.W3 = o.b2 + kMlpHidden;
    o.b3 = o.W3 + kMlpOut * kMlpHidden;
    o.total = o.b3 + kMlpOut;
    return o;
}
cudaError_t mlp_forward(const float* params, const float* x, int B, float* z1, float* a1, float* z2, float* a2,
                        float* y, cudaStream_t s);
// Loss of (y, t) into *loss, dL/dy into dy and every parameter gradient into grad.
cudaError_t mlp_backward(const float* params, const float* x, const float* t, int B, const float* z1,
                         const float* a1, const float* z2, const float* a2, const float* y, float* dy, float* dz2,
                         float* dz1, float* grad, float* loss, cudaStream_t s);
cudaError_t mlp_adam(float* p, const float* g, float* m, float* v, int n, float lr, int step, cudaStream_t s);
cudaError_t mlp_gather_norm(const float* src, const int* idx, int B, int C, const float* mean, const float* stdv,
                            float* dst, cudaStream_t s);
cudaError_t mlp_col_stats(const float* X, int n, int C, float* mean, float* stdv, cudaStream_t s);
cudaError_t launch_features(const Inst* in, const InstIO* io, int batch, int k, int rows_by_user, float* feat,
                            cudaStream_t s);
cudaError_t launch_targets(const Inst* in, int batch, int n_terms, float* tgt, cudaStream_t s);
cudaError_t launch_assemble_low(const Inst* in, int batch, int k, cudaStream_t s);
// The network's mu proposal (and, with use_order, the instance's expansion cut at the
// proposed order times margin, rounded up to whole giant steps).
cudaError_t launch_learned_mu(const Inst* in, int batch, const float* y, const float* norm, int n_terms,
                              int k, int m, int use_order, double margin, cudaStream_t s);
cudaError_t launch_poly_width(const Inst* in, int batch, const Shape& sh, const double* ct, cudaStream_t s);
cudaError_t launch_learned_check(const Inst* in, const InstIO* io, int batch, int round, int max_rounds,
                                 double tol, int is64, int* active_count, cudaStream_t s);

// ------------------------------------------------------------------ coef.cu
cudaError_t launch_cos_table(int M, double* ct, cudaStream_t s);
cudaError_t launch_dos_weights(const Inst* in, int batch, const Shape& sh, const double* ct, cudaStream_t s);
cudaError_t launch_bisect(const Inst* in, const InstIO* io, int batch, const Shape& sh, const double* ct,
                          int max_iter, int start_mu0, cudaStream_t s);
cudaError_t launch_set_mu(const Inst* in, const InstIO* io, int batch, cudaStream_t s);
cudaError_t launch_coefficients(const Inst* in, const InstIO* io, int batch, const Shape& sh,
                                const double* ct, int with_poly_trace, cudaStream_t s, int* launches);
cudaError_t launch_contract(const Inst* in, Work we, Work wct, Work wsym, const Shape& sh, cudaStream_t s, int* dbg);
// g -> the paper's power-basis coefficients d (in place), for the Horner evaluation.
cudaError_t launch_g_to_d(const Inst* in, int batch, const Shape& sh, cudaStream_t s);

// ----------------------------------------------------------- gemm_f64.cu / gemm_tc.cu
int64_t f64_tiles(int64_t np);
cudaError_t launch_gemm_f64(const Step* steps, int nsteps, const Inst* in, const InstIO* io, Work wt,
                            cudaStream_t s);

constexpr int kMaxBuckets = 16;   // tensor maps per grouped launch
int64_t tc_tiles(int64_t np, int tile_n);
int tc_planes(int prec);
// 5-D tensor map over the planes of every slot of every instance of one bucket:
// (column, row, plane, slot, instance), 16-bit elements: boxes of 32 columns x 128 rows with
// 64-byte swizzle (K-major operand tiles) or, with mn, 64 columns x 32 rows with 128-byte
// swizzle (MN-major operand tiles).
bool tc_make_map(void* map128, const void* planes0, int64_t np, int nplanes, int nslots, int count,
                 int64_t slot_bytes, int64_t inst_bytes, bool fp16, std::string* err, bool mn);
// Grouped split-precision product over instances [i0, i1) (sorted by tile count, buckets
// [b0, b0 + nb) with maps: 256 bytes per bucket, its K-major then its MN-major tensor map),
// tile_n = 256 or 128 output columns per tile.
// ctas = CTAs per SM (2 only with tile_n = 128). sym = 0 computes every tile of the full
// product (fo_recurrence_product only), 1 the tiles on and above the diagonal of a symmetric
// product over fully stored planes, 2 the same over planes stored as upper 128-blocks.
// drain = TMEM drain warps (8, or 16 with 256-wide tiles).
// persist = 1: the persistent kernel (tile_n = 128; one CTA per SM walks the tiles, with
// separate epilogue warps overlapping each tile's epilogue with the next tile's products).
cudaError_t tc_gemm(int prec, int tile_n, int ctas, int drain, const Step* steps, int nsteps, const Inst* in, const InstIO* io,
                    const int* pre, int i0, int i1, int tile0, int tiles, const void* maps, int b0,
                    int nb, int* err_flag, cudaStream_t s, std::string* err, int sym = 1, int persist = 0);
// A chain of dependent symmetric products (ChainList) over instances [i0, i1) in one launch,
// windows of consecutive instances holding at least `win_tiles` tiles per step each (0: one
// window). counters: 1 + (i1 - i0) ints of device scratch, zeroed here on `s`.
cudaError_t tc_chain(int prec, int tile_n, int ctas, int drain, const Step* steps, int nsteps, const Inst* in,
                     const InstIO* io, const int* pre_dev, const int* pre_host, int i0, int i1, const void* maps,
                     int b0, int nb, int* err_flag, int* counters, int win_tiles, cudaStream_t s, std::string* err,
                     int sym);
// Tiles of the full (non-symmetric) product.
inline int64_t tc_tiles_full(int64_t np, int tile_n) { return (np / 128) * ((np + tile_n - 1) / tile_n); }

}  // namespace fo
