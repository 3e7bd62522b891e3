// Bandwidth-bound kernels of the solver: per-call setup, spectral bounds, scaling and plane
// splitting, traces, Frobenius inner products (moments) and the output copy. Every kernel
// covers the whole batch in one launch (see internal.cuh for the block-to-instance maps).
//
// All reductions are deterministic: fixed per-thread order, warp shuffles, a fixed tree in
// shared memory, and per-block partials summed in block order by a final kernel.
#include <cstring>

#include <cuda.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "exactsum.h"
#include "fpbits.h"
#include "internal.cuh"

namespace fo {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum in a fixed order; every thread gets the result. blockDim.x <= 1024.
__device__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < nw ? sh[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

// ---------------------------------------------------------------- per-call setup
constexpr int kIoChunk = 64;
struct IoChunk {
    InstIO io[kIoChunk];
    int count, first;
};

__global__ void k_set_io(const IoChunk p, InstIO* d_io, const Inst* insts) {
    const int j = threadIdx.x;
    if (j >= p.count) return;
    const int i = p.first + j;
    d_io[i] = p.io[j];
    DevResult* r = insts[i].res;
    r->bounds[0] = r->bounds[1] = 0.0;
    r->mu = p.io[j].mu;
    r->trace = r->frob2 = r->trace_poly = 0.0;
    r->iters = 0;
    r->status = FO_OK;
    r->nonfinite = 0;
    r->learned_ok = 0;
    r->active = 1;
    r->evals = 0;
    r->mu_lo = r->mu_hi = 0.0;
    r->mu0 = r->mu_prev = r->tr_prev = 0.0;
    r->order = 0.0;
    r->kt_eff = 0.0;
    r->trace_raw = r->gamma = r->proj = 0.0;
    r->fixed = 0;
    r->m_eff = r->n_eff = 0;
}

// ------------------------------------------------------------------ Gershgorin bounds
// One warp per row: r_i = sum_{j != i} |h_ij| summed exactly (lane-strided 128-bit
// fixed-point sums merged by a butterfly, rounded to float64 once: csrc/exactsum.h; the
// float64 adds it replaces bound the kernel on this GPU's narrow float64 pipe), lo_i = h_ii -
// r_i, hi_i = h_ii + r_i; per-block (min lo, max hi, any non-finite).
__global__ void __launch_bounds__(32 * kGershRows) k_gershgorin_rows(const Inst* __restrict__ insts,
                                                                     const InstIO* __restrict__ io,
                                                                     Work wg, double* part) {
    const int b = blockIdx.x;
    const int i = find_inst(wg.pre, 0, wg.count, b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = insts[i].n, ld = io[i].ldh;
    const double* H = io[i].H;
    const int64_t row = (int64_t)(b - wg.pre[i]) * kGershRows + warp;
    double lo = INFINITY, hi = -INFINITY;
    int bad = 0;
    if (row < n) {
        const unsigned long long* r = reinterpret_cast<const unsigned long long*>(H + row * ld);
        XAcc acc{0, 0, 0};
        double d = 0.0;
        // four loads per lane in flight
        int64_t j = lane;
        for (; j + 96 < n; j += 128) {
            uint64_t v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldg(r + j + 32 * u);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool fin = ((v[u] >> 52) & 0x7ff) != 0x7ff;
                bad |= !fin;
                if (j + 32 * u == row) d = __longlong_as_double((long long)v[u]);
                else if (fin) xacc_add_abs(acc, v[u]);
            }
        }
        for (; j < n; j += 32) {
            const uint64_t v = __ldg(r + j);
            const bool fin = ((v >> 52) & 0x7ff) != 0x7ff;
            bad |= !fin;
            if (j == row) d = __longlong_as_double((long long)v);
            else if (fin) xacc_add_abs(acc, v);
        }
        for (int o = 16; o > 0; o >>= 1) {
            XAcc other;
            other.lo = __shfl_xor_sync(0xffffffffu, acc.lo, o);
            other.hi = __shfl_xor_sync(0xffffffffu, acc.hi, o);
            other.e = __shfl_xor_sync(0xffffffffu, acc.e, o);
            xacc_merge(acc, other);
        }
        const double s = xacc_to_double(acc);
        d = warp_sum(d);
        lo = d - s;
        hi = d + s;
    }
    bad = __any_sync(0xffffffffu, bad);
    __shared__ double slo[kGershRows], shi[kGershRows];
    __shared__ int sbad[kGershRows];
    if (lane == 0) { slo[warp] = lo; shi[warp] = hi; sbad[warp] = bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double l = slo[0], h = shi[0];
        int bd = sbad[0];
        for (int w = 1; w < kGershRows; ++w) {
            l = fmin(l, slo[w]);
            h = fmax(h, shi[w]);
            bd |= sbad[w];
        }
        part[3 * (int64_t)b] = l;
        part[3 * (int64_t)b + 1] = h;
        part[3 * (int64_t)b + 2] = bd ? 1.0 : 0.0;
    }
}

// One block per instance: reduce its partials [pre[i], pre[i+1]).
__global__ void k_gershgorin_final(const Inst* __restrict__ insts, Work wg, const double* part) {
    __shared__ double slo[32], shi[32];
    __shared__ int sbad[32];
    const int i = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double lo = INFINITY, hi = -INFINITY;
    int bad = 0;
    for (int q = wg.pre[i] + threadIdx.x; q < wg.pre[i + 1]; q += blockDim.x) {
        lo = fmin(lo, part[3 * (int64_t)q]);
        hi = fmax(hi, part[3 * (int64_t)q + 1]);
        bad |= part[3 * (int64_t)q + 2] != 0.0;
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) { slo[warp] = lo; shi[warp] = hi; sbad[warp] = bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) {
            lo = fmin(lo, slo[w]);
            hi = fmax(hi, shi[w]);
            bad |= sbad[w];
        }
        if (!(hi - lo > 1e-12 * fmax(1.0, fmax(fabs(lo), fabs(hi))))) {
            const double c = 0.5 * (lo + hi);
            lo = c - 1.0;
            hi = c + 1.0;
        }
        DevResult* r = insts[i].res;
        r->bounds[0] = lo;
        r->bounds[1] = hi;
        r->nonfinite = bad;
        r->status = bad ? FO_ERR_NONFINITE : FO_OK;
    }
}

// Given bounds (InstIO emin/emax) or bounds copied from device memory (bounds_src).
__global__ void k_bounds_given(const Inst* __restrict__ insts, const InstIO* __restrict__ io, int batch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    DevResult* r = insts[i].res;
    if (io[i].bounds_src) {
        r->bounds[0] = io[i].bounds_src[0];
        r->bounds[1] = io[i].bounds_src[1];
    } else {
        r->bounds[0] = io[i].emin;
        r->bounds[1] = io[i].emax;
    }
    r->nonfinite = 0;
    r->status = FO_OK;
}

__global__ void k_export_bounds(const DevResult* res, double* out3) {
    out3[0] = res->bounds[0];
    out3[1] = res->bounds[1];
    out3[2] = res->nonfinite ? 1.0 : 0.0;
}

// ------------------------------------------------------------- scaling and splitting

__device__ __forceinline__ uint16_t bf16_bits(__nv_bfloat16 h) {
    return *reinterpret_cast<uint16_t*>(&h);
}
__device__ __forceinline__ uint16_t f16_bits(__half h) { return *reinterpret_cast<uint16_t*>(&h); }

// Store v (float32) and its split planes. BF16: v = h0 + h1 + h2 with each remainder
// computed exactly in float32. FP16: the value is first multiplied by pscale (a power of
// two) so that the entries use the fp16 normal range; v*pscale = h0 + h1.
__device__ __forceinline__ void store_split(float v, float* x, uint16_t* p, int64_t pstride,
                                            int planes, int fp16, float pscale) {
    if (x) *x = v;
    if (planes <= 0) return;
    if (!fp16) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v);
        p[0] = bf16_bits(h0);
        if (planes > 1) {
            const float r1 = v - __bfloat162float(h0);
            const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
            p[pstride] = bf16_bits(h1);
            if (planes > 2) {
                const float r2 = r1 - __bfloat162float(h1);
                p[2 * pstride] = bf16_bits(__float2bfloat16_rn(r2));
            }
        }
    } else {
        const float vs = v * pscale;
        const __half h0 = __float2half_rn(vs);
        p[0] = f16_bits(h0);
        if (planes > 1) p[pstride] = f16_bits(__float2half_rn(vs - __half2float(h0)));
    }
}

// X = (2H - (emin+emax) I) / (emax - emin) into slot 0 (np x np, zero border), built from
// the upper triangle of H only, so that X is exactly symmetric. One block per 32 x 32 tile
// (bi, bj), bj >= bi, of one instance: the H tile is staged in shared memory, each of its
// entries is scaled once (float64; off the diagonal as h * (2 / (emax - emin)), which equals
// (2h) / (emax - emin) rounded once since both factors of 2 are exact) and the scaled tile is
// written to X at (bi, bj) and, transposed, at (bj, bi). Output float64, or float32 + planes
// (the float64 pipe of this GPU is narrow: one multiply per entry; the rounding to float32 is
// done with integer operations).
__global__ void __launch_bounds__(256) k_scale_sym(const Inst* __restrict__ insts,
                                                   const InstIO* __restrict__ io, Work ws,
                                                   const Shape sh, int* dbg) {
    __shared__ double tile[32][33];
    __shared__ float tf[32][33];
    const int i = find_inst(ws.pre, 0, ws.count, blockIdx.x);
    const int64_t n = insts[i].n, np = insts[i].np, ld = io[i].ldh;
    const double* H = io[i].H;
    const DevResult* res = insts[i].res;
    const int tn = (int)(np / 32);
    int bi, bj;
    upper_tile(blockIdx.x - ws.pre[i], tn, bi, bj);
    // the scale factors once per block: a float64 division per thread would cost more than
    // the block's multiplies on this GPU's narrow float64 pipe
    __shared__ double s_par[3];
    if (threadIdx.x == 0) {
        const double ea = res->bounds[0], eb = res->bounds[1];
        s_par[0] = 1.0 / (eb - ea);
        s_par[1] = 2.0 * s_par[0];
        s_par[2] = ea + eb;
    }
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int ry = ty; ry < 32; ry += 8) {
        const int64_t r = (int64_t)bi * 32 + ry, c = (int64_t)bj * 32 + tx;
        tile[ry][tx] = (r < n && c < n) ? H[r * ld + c] : 0.0;
    }
    __syncthreads();
    const double inv = s_par[0], inv2 = s_par[1], csum = s_par[2];
    // each thread scales the entries it loaded (the lower half of a diagonal tile is never
    // read: it is written from the upper half); the diagonal's formula only in diagonal tiles
    // (a block-uniform test, so that the other tiles carry no float64 work for it)
    for (int ry = ty; ry < 32; ry += 8) {
        const int64_t r = (int64_t)bi * 32 + ry, c = (int64_t)bj * 32 + tx;
        const bool in = r < n && c < n && (bi != bj || tx >= ry);
        const bool dg = bi == bj && r == c;
        if (sh.is64) {
            double v = 0.0;
            if (in) v = dg ? (2.0 * tile[ry][tx] - csum) * inv : tile[ry][tx] * inv2;
            tile[ry][tx] = v;
        } else {
            // float32 of the exact product in integer operations (the float64 multiply was
            // this kernel's bound on the narrow float64 pipe)
            float f = 0.0f;
            if (in) f = dg ? narrow_f64((2.0 * tile[ry][tx] - csum) * inv) : mul_rn_f32(tile[ry][tx], inv2);
            tf[ry][tx] = f;
        }
    }
    __syncthreads();
    char* slot = insts[i].slots;
    double* X64 = reinterpret_cast<double*>(slot);
    float* X32 = reinterpret_cast<float*>(slot);
    uint16_t* P16 = reinterpret_cast<uint16_t*>(slot + 4 * np * np);
    for (int ry = ty; ry < 32; ry += 8) {
        // (bi*32 + ry, bj*32 + tx); in a diagonal tile the lower half mirrors the upper
        // upper-block storage keeps the transposed tile below the diagonal inside the diagonal
        // 128-block only (a lower 128-block is read as the transpose of its upper counterpart)
        const bool lower = bi != bj && (!sh.ublk || bi * 32 / kPad == bj * 32 / kPad);
        for (int pass = 0; pass < (lower ? 2 : 1); ++pass) {
            int64_t r, c;
            int tr, tc;   // entry of the scaled tile
            if (pass == 0) {
                r = (int64_t)bi * 32 + ry;
                c = (int64_t)bj * 32 + tx;
                const bool mir = bi == bj && tx < ry;
                tr = mir ? tx : ry;
                tc = mir ? ry : tx;
            } else {
                r = (int64_t)bj * 32 + ry;
                c = (int64_t)bi * 32 + tx;
                tr = tx;
                tc = ry;
            }
            const int64_t idx = r * np + c;
            if (!FO_CHK(dbg, r < np && c < np, 201, r, c)) continue;
            if (sh.is64) X64[idx] = tile[tr][tc];
            // below the diagonal only the planes are kept (float32 masters: on and above it)
            else store_split(tf[tr][tc], r <= c ? X32 + idx : nullptr, P16 + idx, np * np, sh.planes, sh.fp16,
                             sh.pscale_t);
        }
    }
}

__global__ void k_pack_f32(const float* __restrict__ A, int64_t n, int64_t lda, char* slot, int64_t np,
                           int planes, int fp16, float pscale) {
    const int64_t total = np * np;
    float* x = reinterpret_cast<float*>(slot);
    uint16_t* p = reinterpret_cast<uint16_t*>(slot + 4 * total);
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / np, col = idx - r * np;
        const float v = (r < n && col < n) ? A[r * lda + col] : 0.0f;
        store_split(v, x + idx, p + idx, total, planes, fp16, pscale);
    }
}

// ----------------------------------------------------------------------- traces
// diag[s] = sum_{r<n} slot_s[r, r] (float64); block (s, instance).
__global__ void k_diag_sums(const Inst* __restrict__ insts, int is64) {
    __shared__ double sh[33];
    const Inst& in = insts[blockIdx.y];
    if (!in.res->active) return;
    const int64_t n = in.n, np = in.np;
    const char* slot = in.slots + in.slot_bytes * blockIdx.x;
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        s += is64 ? reinterpret_cast<const double*>(slot)[r * np + r]
                  : (double)reinterpret_cast<const float*>(slot)[r * np + r];
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) in.diag[blockIdx.x] = s;
}

// --------------------------------------------------------- Frobenius inner products
// <S_{giant0+g}, S_{baby0+b}>_F of one instance. Every matrix is symmetric, so the product is
// the diagonal sum plus twice the strict upper triangle: only the chunks (kChunk consecutive
// entries of one row) on or above the diagonal are read. A block covers kGChunks consecutive
// upper chunks. They are copied kCPS chunks at a time into a kGStages-deep shared-memory ring
// by cp.async (16 bytes per copy, no register staging; each thread's copy addresses are
// fixed up front and only offset per chunk), matrix-major (row s of a chunk holds the chunk
// of matrix s, rows padded by 16 bytes), so that kGStages - 1 stages are in flight while one
// is multiplied; one barrier per stage separates its consumption from the refill of the
// stage it frees. Each warp owns up to TPW tiles of TG x TB (giant, baby) pairs; a lane reads
// 16-byte vectors of TG + TB rows and accumulates TG x TB x (16 / sizeof(T)) products per
// step (float32: packed FMAs, even and odd entries in the two lanes). One 5 x 5, 4 x 5 or
// 5 x 4 tile per warp where the pairs fit 16 warps, else two 4 x 4 tiles per warp (see
// gram_shape): a larger tile reads each staged vector from shared memory fewer times per
// product and leaves each warp more independent loads in flight, which is what bounds this
// kernel (shared-load latency). Chunks right of the
// diagonal weigh the baby entries by 1 (the factor 2 of the strict upper triangle is applied
// once at the end); the diagonal chunk of a row weighs them by 1, 1/2 or 0 right of, on or
// left of the diagonal. Every lane sums at most kGChunks * kChunk / 32 products per pair in
// T; lanes are combined by shuffles in T and blocks by the float64 partial sums (k_sum_partials).
constexpr int kChunkBytes = 512;    // one chunk of one matrix: 128 float32 / 64 float64
constexpr int kGChunks = 64;        // chunks per block
constexpr int kCPS = 2;             // chunks per stage
constexpr int kGStages = 4;         // shared-memory ring depth (stages)
constexpr int kMaxRows = 48;        // staged rows (giant and baby groups, padded)
constexpr int kGramThreads = 512;   // largest block: 16 warps
constexpr int kGramMinThreads = 256;
// 16-byte copies per thread and chunk: staged rows x (kChunkBytes / 16) vectors / threads
constexpr int kGLoads = (kMaxRows * (kChunkBytes / 16) + kGramMinThreads - 1) / kGramMinThreads;

// Threads of a block for ntiles (giant, baby) tiles: tpw tiles per warp, at least 8 warps.
__host__ __device__ inline int gram_threads(int ntiles, int tpw) {
    int w = (ntiles + tpw - 1) / tpw;
    if (w < kGramMinThreads / 32) w = kGramMinThreads / 32;
    return 32 * w;
}

// Upper chunks of an np x np matrix: row r holds chunks floor(r / kc) .. np / kc - 1.
__host__ __device__ inline int64_t upper_chunks(int64_t np, int kc) {
    const int64_t cpr = np / kc;
    return (int64_t)kc * cpr * (cpr + 1) / 2;
}

template <typename T, int TG, int TB, int TPW>
__global__ void __launch_bounds__(kGramThreads, 1) k_gram(const Inst* __restrict__ insts, Work wgr, int giant0,
                                                          int ngiant, int baby0, int nbaby) {
    constexpr int NP = TG * TB;                // pairs per tile
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int kChunk = kChunkBytes / (int)sizeof(T);      // entries per chunk
    constexpr int V = 16 / sizeof(T);          // elements per 16-byte vector
    constexpr int RS = kChunk + V;             // row stride (elements)
    constexpr int VPR = kChunk / V;            // vectors per row
    const int i = find_inst(wgr.pre, 0, wgr.count, blockIdx.x);
    const Inst& in = insts[i];
    if (!in.res->active) return;
    const int lb = blockIdx.x - wgr.pre[i];
    const char* base = in.slots;
    const int64_t slot_bytes = in.slot_bytes;
    const int64_t np = in.np;
    const int64_t cpr = np / kChunk;                  // chunks per row
    const int64_t nchunks = upper_chunks(np, kChunk);
    const int64_t c0 = (int64_t)lb * kGChunks;
    const int64_t c1 = c0 + kGChunks < nchunks ? c0 + kGChunks : nchunks;
    const int ngq = (ngiant + TG - 1) / TG, nbq = (nbaby + TB - 1) / TB;
    const int nrows = TG * ngq + TB * nbq;
    const int ntiles = ngq * nbq;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int chunk_elems = nrows * RS;
    const int stage_elems = kCPS * chunk_elems;
    T* ring = reinterpret_cast<T*>(smem_raw);

    // (row, chunk of the row) of upper chunk c0; rows of band b (kChunk rows) hold cpr - b
    int64_t row = 0, cc = 0;
    if (c0 < c1) {
        int64_t b = 0, cum = 0;
        while (cum + (int64_t)kChunk * (cpr - b) <= c0) {
            cum += (int64_t)kChunk * (cpr - b);
            ++b;
        }
        const int64_t off = c0 - cum, per = cpr - b;
        row = (int64_t)kChunk * b + off / per;
        cc = b + off % per;
    }
    auto advance = [&](int64_t& r, int64_t& c) {
        if (++c == cpr) {
            ++r;
            c = r / kChunk;
        }
    };
    // slot of staged row srow, or -1 for the padding rows of a partial quad
    auto slot_of = [&](int srow) -> int {
        if (srow < TG * ngq) return srow < ngiant ? giant0 + srow : -1;
        const int bb = srow - TG * ngq;
        return bb < nbaby ? baby0 + bb : -1;
    };
    // this thread's copies: source at chunk (0, 0) and shared-memory offset in a chunk
    const char* gsrc[kGLoads];
    int sdst[kGLoads];
#pragma unroll
    for (int j = 0; j < kGLoads; ++j) {
        const int q = threadIdx.x + j * (int)blockDim.x;
        gsrc[j] = nullptr;
        sdst[j] = 0;
        if (q < nrows * VPR) {
            const int srow = q / VPR, ev = (q % VPR) * V;
            const int slot = slot_of(srow);
            sdst[j] = srow * RS + ev;
            if (slot >= 0) gsrc[j] = base + slot_bytes * slot + (int64_t)ev * (int64_t)sizeof(T);
        }
    }
    // the padding rows hold zeros in every stage, written once
    for (int q = threadIdx.x; q < kGStages * kCPS * nrows * VPR; q += blockDim.x) {
        const int st = q / (nrows * VPR), w = q % (nrows * VPR);
        const int srow = w / VPR, ev = (w % VPR) * V;
        if (slot_of(srow) < 0)
            *reinterpret_cast<float4*>(ring + st * chunk_elems + srow * RS + ev) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int64_t nch = c1 - c0;
    const int nst = (int)((nch + kCPS - 1) / kCPS);
    int64_t ir = row, ic = cc, issued = 0;   // next chunk to copy
    auto issue_stage = [&](int st) {
        T* dst = ring + (st % kGStages) * stage_elems;
#pragma unroll
        for (int u = 0; u < kCPS; ++u) {
            if (issued < nch) {
                const int64_t off = (ir * np + ic * kChunk) * (int64_t)sizeof(T);
#pragma unroll
                for (int j = 0; j < kGLoads; ++j)
                    if (gsrc[j]) cp_async16(dst + u * chunk_elems + sdst[j], gsrc[j] + off);
                advance(ir, ic);
                ++issued;
            }
        }
    };

    T acc[TPW][NP];        // float64 sums
    float2 acc2[TPW][NP];   // float32 sums of the even / odd entries
#pragma unroll
    for (int t = 0; t < TPW; ++t)
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            acc[t][q] = T(0);
            acc2[t][q] = make_float2(0.0f, 0.0f);
        }

    // shared-memory offsets of this warp's tiles (-1: none)
    int toff_g[TPW], toff_b[TPW];
#pragma unroll
    for (int t = 0; t < TPW; ++t) {
        const int tile = warp + t * nwarps;
        toff_g[t] = tile < ntiles ? TG * (tile / nbq) * RS : -1;
        toff_b[t] = tile < ntiles ? (TG * ngq + TB * (tile % nbq)) * RS : -1;
    }
#pragma unroll
    for (int s = 0; s < kGStages - 1; ++s) {
        if (s < nst) issue_stage(s);
        cp_async_commit();
    }
    int64_t done = 0;
    for (int s = 0; s < nst; ++s) {
        cp_async_wait<kGStages - 2>();   // this thread's copies of stage s have landed
        __syncthreads();                 // everyone's have; the ring slot of stage s - 1 is free
        if (s + kGStages - 1 < nst) issue_stage(s + kGStages - 1);
        cp_async_commit();
        const T* stage_base = ring + (s % kGStages) * stage_elems;
        // chunks of this stage: how many, and which one holds a diagonal entry at (row, col)
        int nu = 0;
        int64_t drow[kCPS], dcol0[kCPS];
#pragma unroll
        for (int u = 0; u < kCPS; ++u) {
            drow[u] = -1;
            dcol0[u] = 0;
            if (done < nch) {
                if (cc == row / kChunk) {
                    drow[u] = row;
                    dcol0[u] = cc * kChunk;
                }
                advance(row, cc);
                ++done;
                ++nu;
            }
        }
#pragma unroll
        for (int t = 0; t < TPW; ++t) {
            if (toff_g[t] < 0) break;                   // uniform across the warp
#pragma unroll
            for (int u = 0; u < kCPS; ++u) {
                if (u >= nu) break;
                const T* g0 = stage_base + u * chunk_elems + toff_g[t];
                const T* b0 = stage_base + u * chunk_elems + toff_b[t];
                for (int e = lane * V; e < kChunk; e += 32 * V) {
                    T gv[TG][V], bv[TB][V];
#pragma unroll
                    for (int a = 0; a < TG; ++a)
                        *reinterpret_cast<float4*>(gv[a]) = *reinterpret_cast<const float4*>(g0 + a * RS + e);
#pragma unroll
                    for (int b = 0; b < TB; ++b)
                        *reinterpret_cast<float4*>(bv[b]) = *reinterpret_cast<const float4*>(b0 + b * RS + e);
                    if (drow[u] >= 0) {
                        // the entries left of the diagonal are not maintained (the float32
                        // masters are kept on and above it only): select, never multiply
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            const int64_t col = dcol0[u] + e + v;
#pragma unroll
                            for (int b = 0; b < TB; ++b)
                                bv[b][v] = col > drow[u] ? bv[b][v] : (col == drow[u] ? T(0.5) * bv[b][v] : T(0));
#pragma unroll
                            for (int a = 0; a < TG; ++a) gv[a][v] = col >= drow[u] ? gv[a][v] : T(0);
                        }
                    }
                    if constexpr (sizeof(T) == 4) {
#pragma unroll
                        for (int a = 0; a < TG; ++a)
#pragma unroll
                            for (int b = 0; b < TB; ++b) {
                                float2& s2 = acc2[t][TB * a + b];
                                s2 = __ffma2_rn(make_float2(gv[a][0], gv[a][1]), make_float2(bv[b][0], bv[b][1]), s2);
                                s2 = __ffma2_rn(make_float2(gv[a][2], gv[a][3]), make_float2(bv[b][2], bv[b][3]), s2);
                            }
                    } else {
#pragma unroll
                        for (int a = 0; a < TG; ++a)
#pragma unroll
                            for (int b = 0; b < TB; ++b)
#pragma unroll
                                for (int v = 0; v < V; ++v)
                                    acc[t][TB * a + b] = fma(gv[a][v], bv[b][v], acc[t][TB * a + b]);
                    }
                }
            }
        }
    }
    cp_async_wait<0>();
    const int npairs = ngiant * nbaby;
    double* partials = in.gpart;
#pragma unroll
    for (int t = 0; t < TPW; ++t) {
        const int tile = warp + t * nwarps;
        if (tile >= ntiles) break;
        const int tg = tile / nbq, tb = tile % nbq;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int g = TG * tg + q / TB, b = TB * tb + q % TB;
            if constexpr (sizeof(T) == 4) {
                // float32 tree over the lanes: the float64 pipe of this GPU retires about two
                // lane operations per clock and SM, so a float64 tree per pair would cost more
                // than the block's loads; one conversion per pair on lane 0
                const float2 pr = acc2[t][q];
                float v = pr.x + pr.y;
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0 && g < ngiant && b < nbaby) partials[(int64_t)lb * npairs + g * nbaby + b] = 2.0 * (double)v;
            } else {
                double v = 2.0 * (double)acc[t][q];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0 && g < ngiant && b < nbaby) partials[(int64_t)lb * npairs + g * nbaby + b] = v;
            }
        }
    }
}

// Frobenius products of float32 masters, the same unit partials as k_gram<float>: one
// partial per (instance, kGChunks upper chunks, pair), written as 2 x the unit's sum with
// the diagonal entry weighed 1/2. Persistent blocks (one per SM) take the units of one
// group of tensor-map buckets round-robin. One thread of warp ncons loads each chunk (128
// consecutive entries of one matrix row) of a stage with two TMA copies, a box of 128
// columns x 1 row x ngiant slots from the giant matrices and one of nbaby slots from the
// baby matrices (4-D tensor maps over (column, row, slot, instance) of the float32
// masters): two copies per chunk instead of one per matrix, since the copy engine's cost
// per copy, not the bytes, bounded a ring fed by per-matrix bulk copies. The ring is S
// stages of CPS chunks, laid out (stage, chunk, staged row, entry) with padding rows zero;
// the copy thread publishes each chunk's diagonal position before it arms the stage's
// `full` mbarrier, and the consumer warps release a stage through `empty`. Consumer warp w
// owns the (giant, baby) tile w / H of TG x TB pairs and every H-th 32-entry group of each
// stage: lane l multiplies entry l of the group in the TG giant rows with the same entry of
// the TB baby rows, two giant rows per packed FMA (the baby value in both halves), so one
// staged word feeds TB / 2 or TG packed FMAs. At the end of a unit a warp's sums are
// reduced over its lanes by halving exchanges (each lane keeps half of what it holds, five
// times: about 124 shuffles instead of 5 per sum), the H warps of a tile are added through
// shared memory and the tile's first warp writes the partials. Every wait is bounded; a
// wait that gives up sets the block's abort flag and the device error flag, the consumers
// keep to the control flow without computing (so that every named barrier is reached), and
// the copy thread waits, bounded, for the copies it issued before the block exits.
constexpr int kRMaxStages = 6;                     // ring depth at most
constexpr int kRSmemBudget = 200 * 1024;           // ring bytes at most
constexpr int kRMaxCPS = 8;                        // chunks per stage at most
constexpr int kRMaxCons = 8;                       // consumer warps
constexpr int kRThreads = 32 * (kRMaxCons + 1);
constexpr int kRMaxRows = 64;                      // staged rows (padded groups)
constexpr int kRChunk = kChunkBytes / 4;           // float32 entries per chunk

struct GramMaps {
    CUtensorMap g[kMaxBuckets];   // boxes of 128 columns x 1 row x ngiant slots
    CUtensorMap b[kMaxBuckets];   // boxes of 128 columns x 1 row x nbaby slots
};

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// (row, chunk of the row) of upper chunk c of an np x np matrix cut into kc-entry chunks
__device__ __forceinline__ void upper_chunk_pos(int64_t c, int64_t np, int kc, int& row, int& cc) {
    const int64_t cpr = np / kc;
    int64_t b = 0, cum = 0;
    while (cum + (int64_t)kc * (cpr - b) <= c) {
        cum += (int64_t)kc * (cpr - b);
        ++b;
    }
    const int64_t off = c - cum, per = cpr - b;
    row = (int)((int64_t)kc * b + off / per);
    cc = (int)(b + off % per);
}

// One halving exchange: lanes with `BIT` set keep v[HS..2HS), the others v[0..HS), each
// adding its partner's copy of the half it keeps (lane ^ BIT); the kept half moves to v[0..HS).
template <int HS, int BIT>
__device__ __forceinline__ void halve_lanes(float (&v)[128], int lane) {
    const bool up = (lane & BIT) != 0;
#pragma unroll
    for (int q = 0; q < HS; ++q) {
        const float send = up ? v[q] : v[q + HS];
        const float keep = up ? v[q + HS] : v[q];
        v[q] = keep + __shfl_xor_sync(0xffffffffu, send, BIT);
    }
}

template <int TG, int TB>
__global__ void __launch_bounds__(kRThreads, 1)
    k_gram_ring(const __grid_constant__ GramMaps maps, const Inst* __restrict__ insts, Work wgr, int u0, int u1,
                int b0, int giant0, int ngiant, int baby0, int nbaby, int H, int S, int CPS, int* err) {
    static_assert(TG % 2 == 0 && TG * TB <= 128, "tile");
    constexpr int NP = TG * TB;
    constexpr int RS = kRChunk;                         // row stride of the ring (floats)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ngq = (ngiant + TG - 1) / TG, nbq = (nbaby + TB - 1) / TB;
    const int R = TG * ngq + TB * nbq;                  // staged rows; padding rows stay zero
    const int ncons = ngq * nbq * H;
    const int chunk_floats = R * RS;
    const int stage_floats = CPS * chunk_floats;
    // the ring starts on a 1024-byte boundary (every TMA destination is then 512-byte aligned)
    unsigned char* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    float* ring = reinterpret_cast<float*>(sm);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)S * stage_floats * 4);
    uint64_t* empty = full + kRMaxStages;
    float* red = reinterpret_cast<float*>(empty + kRMaxStages);   // [ncons][32 lanes][4]
    // per stage and chunk: (row, first column) when the chunk holds its row's diagonal entry
    // (the row's first upper chunk), else row -1
    __shared__ int2 s_diag[kRMaxStages][kRMaxCPS];
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bro0 = TG * ngq;                          // first baby row of a chunk
    if (threadIdx.x == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], ncons);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int q = threadIdx.x; q < S * stage_floats; q += blockDim.x) {
        const int j = (q / RS) % R;
        if ((j >= ngiant && j < bro0) || j >= bro0 + nbaby) ring[q] = 0.0f;
    }
    __syncthreads();

    const int nreal = ngiant + nbaby;
    volatile int* va = &s_abort;
    // warp-uniform view of the abort flag (lane 0 reads it)
    auto aborted = [&]() -> bool {
        int a = 0;
        if (lane == 0) a = *va;
        return __shfl_sync(0xffffffffu, a, 0) != 0;
    };
    // ring position: slot and the parity of its current use
    int slot = 0;
    uint32_t phase = 0;
    if (warp == ncons) {
        // ---------------------------------------------------------------- copy thread
        if (lane != 0) return;
        int64_t issued = 0;                 // stages whose copies were issued
        bool stop = false;
        for (int u = u0 + blockIdx.x; u < u1 && !stop; u += gridDim.x) {
            const int i = find_inst(wgr.pre, 0, wgr.count, u);
            const Inst& in = insts[i];
            if (!in.res->active) continue;
            const int64_t np = in.np, nchunks = upper_chunks(np, kRChunk);
            const int cpr = (int)(np / kRChunk);
            const int64_t c0 = (int64_t)(u - wgr.pre[i]) * kGChunks;
            const int nch = (int)((c0 + kGChunks < nchunks ? c0 + kGChunks : nchunks) - c0);
            const CUtensorMap* mg = &maps.g[in.bucket - b0];
            const CUtensorMap* mb = &maps.b[in.bucket - b0];
            int row, cc;
            upper_chunk_pos(c0, np, kRChunk, row, cc);
            for (int st = 0; st * CPS < nch; ++st) {
                if (issued >= S && !mbar_wait(&empty[slot], phase ^ 1u, kWaitNs, va)) {
                    *va = 1;
                    atomicExch(err, 1);
                }
                if (*va) {
                    stop = true;
                    break;
                }
                const int nc = nch - st * CPS < CPS ? nch - st * CPS : CPS;
                mbar_expect_tx(&full[slot], (uint32_t)(nc * nreal * kChunkBytes));
                float* dst = ring + (size_t)slot * stage_floats;
                for (int q = 0; q < nc; ++q, dst += chunk_floats) {
                    s_diag[slot][q] = make_int2(cc == row / kRChunk ? row : -1, cc * kRChunk);
                    tma_load_4d(dst, mg, &full[slot], cc * kRChunk, row, giant0, in.in_bucket);
                    tma_load_4d(dst + bro0 * RS, mb, &full[slot], cc * kRChunk, row, baby0, in.in_bucket);
                    if (++cc == cpr) cc = ++row / kRChunk;
                }
                ++issued;
                if (++slot == S) {
                    slot = 0;
                    phase ^= 1u;
                }
            }
        }
        // an aborted block waits for the copies it issued before it exits
        if (*va) {
            for (int64_t g = issued > S ? issued - S : 0; g < issued; ++g)
                mbar_wait(&full[g % S], (uint32_t)(g / S) & 1u, kDrainNs, nullptr);
        }
        return;
    }
    if (warp > ncons) return;

    // -------------------------------------------------------------------- consumers
    const int tile = warp / H, hh = warp % H;
    const int gro = TG * (tile / nbq), bro = bro0 + TB * (tile % nbq);
    float2 acc[TG / 2][TB];
#pragma unroll
    for (int a = 0; a < TG / 2; ++a)
#pragma unroll
        for (int b = 0; b < TB; ++b) acc[a][b] = make_float2(0.0f, 0.0f);
    for (int u = u0 + blockIdx.x; u < u1; u += gridDim.x) {
        const int i = find_inst(wgr.pre, 0, wgr.count, u);
        const Inst& in = insts[i];
        if (!in.res->active) continue;
        const int64_t nchunks = upper_chunks(in.np, kRChunk);
        const int lb = u - wgr.pre[i];
        const int64_t c0 = (int64_t)lb * kGChunks;
        const int nch = (int)((c0 + kGChunks < nchunks ? c0 + kGChunks : nchunks) - c0);
        for (int st = 0; st * CPS < nch; ++st) {
            const bool ok = !aborted() && mbar_wait_warp(&full[slot], phase, kWaitNs, va);
            if (!ok && lane == 0 && !*va) {
                *va = 1;
                atomicExch(err, 1);
            }
            const int nc = nch - st * CPS < CPS ? nch - st * CPS : CPS;
            if (ok) {
                const int sbase = slot * stage_floats;
                const int gi = sbase + gro * RS + lane, bi = sbase + bro * RS + lane;
                for (int q = hh; q < nc * (kRChunk / 32); q += H) {
                    const int off = (q >> 2) * chunk_floats + (q & 3) * 32;   // chunk q / 4, group q % 4
                    float gv[TG], bv[TB];
#pragma unroll
                    for (int a = 0; a < TG; ++a) gv[a] = ring[gi + a * RS + off];
#pragma unroll
                    for (int b = 0; b < TB; ++b) bv[b] = ring[bi + b * RS + off];
                    const int2 dg = s_diag[slot][q >> 2];
                    if (dg.x >= 0) {
                        // left of the diagonal the words are stale: select, never multiply
                        const int col = dg.y + (q & 3) * 32 + lane;
                        const float wb = col > dg.x ? 1.0f : 0.5f;
#pragma unroll
                        for (int b = 0; b < TB; ++b) bv[b] = col >= dg.x ? wb * bv[b] : 0.0f;
#pragma unroll
                        for (int a = 0; a < TG; ++a) gv[a] = col >= dg.x ? gv[a] : 0.0f;
                    }
#pragma unroll
                    for (int b = 0; b < TB; ++b) {
                        const float2 bb = make_float2(bv[b], bv[b]);
#pragma unroll
                        for (int a = 0; a < TG / 2; ++a)
                            acc[a][b] = __ffma2_rn(make_float2(gv[2 * a], gv[2 * a + 1]), bb, acc[a][b]);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
            if (++slot == S) {
                slot = 0;
                phase ^= 1u;
            }
        }

        // unit end: halving exchanges over the lanes; lane l keeps entries base(l) + 0..3
        float v[128];
#pragma unroll
        for (int q = 0; q < 128; ++q) {
            if (q < NP) {
                const float2 pr = acc[(q / TB) / 2][q % TB];
                v[q] = ((q / TB) & 1) ? pr.y : pr.x;
            } else {
                v[q] = 0.0f;
            }
        }
        halve_lanes<64, 16>(v, lane);
        halve_lanes<32, 8>(v, lane);
        halve_lanes<16, 4>(v, lane);
        halve_lanes<8, 2>(v, lane);
        halve_lanes<4, 1>(v, lane);
        const int base = ((lane >> 4) & 1) * 64 + ((lane >> 3) & 1) * 32 + ((lane >> 2) & 1) * 16 +
                         ((lane >> 1) & 1) * 8 + (lane & 1) * 4;
        if (H > 1) {
#pragma unroll
            for (int j = 0; j < 4; ++j) red[(warp * 32 + lane) * 4 + j] = v[j];
            asm volatile("bar.sync 1, %0;" ::"r"(ncons * 32) : "memory");
        }
        if (hh == 0) {
            const int npairs = ngiant * nbaby;
            double* partials = in.gpart + (int64_t)lb * npairs;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float sum = v[j];
                for (int w = 1; w < H; ++w) sum += red[((warp + w) * 32 + lane) * 4 + j];
                const int q = base + j;
                const int ga = gro + q / TB, b = (bro - bro0) + q % TB;
                if (q < NP && ga < ngiant && b < nbaby) partials[ga * nbaby + b] = (double)(2.0f * sum);
            }
        }
        if (H > 1) asm volatile("bar.sync 1, %0;" ::"r"(ncons * 32) : "memory");
#pragma unroll
        for (int a = 0; a < TG / 2; ++a)
#pragma unroll
            for (int b = 0; b < TB; ++b) acc[a][b] = make_float2(0.0f, 0.0f);
    }
}

// gram[out0 + pq] = sum over the instance's blocks of partial pq, in a fixed order; one
// block per (pair, instance), threads strided over the partials.
__global__ void k_sum_partials(const Inst* __restrict__ insts, int npairs, int out0) {
    __shared__ double sh[33];
    const Inst& in = insts[blockIdx.y];
    if (!in.res->active) return;
    const int pq = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < in.gram_blocks; b += blockDim.x) s += in.gpart[(int64_t)b * npairs + pq];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) in.gram[out0 + pq] = s;
}

// tau[0..n_terms) from baby traces diag[0..k) (T_1..T_k), giant traces diag[k + l - 2]
// (T_{lk}, l = 2..m-1) and gram[(l-1)*(k-1) + (i-1)] = <T_{lk}, T_i> (l = 1..m-1,
// i = 1..k-1) through tau_{lk+i} = 2 <T_{lk}, T_i> - tau_{lk-i} (Eq. identity).
// Within one l the k - 1 moments are independent (tau_{lk-i} belongs to the range of l - 1):
// threads take i, the block steps through l (a serial loop of dependent global loads took
// tens of microseconds).
__global__ void k_assemble_moments(const Inst* __restrict__ insts, int k, int m, int n_terms) {
    const Inst& in = insts[blockIdx.x];
    if (!in.res->active) return;
    const double* diag = in.diag;
    const double* gram = in.gram;
    double* tau = in.tau;
    if (threadIdx.x == 0) tau[0] = (double)in.n;
    for (int i = 1 + (int)threadIdx.x; i <= k && i < n_terms; i += blockDim.x) tau[i] = diag[i - 1];
    __syncthreads();
    for (int l = 1; l < m; ++l) {
        const int base = l * k;
        if (base >= n_terms) break;
        if (l >= 2 && threadIdx.x == 0) tau[base] = diag[k + l - 2];
        for (int i = 1 + (int)threadIdx.x; i < k && base + i < n_terms; i += blockDim.x)
            tau[base + i] = 2.0 * gram[(l - 1) * (k - 1) + (i - 1)] - tau[base - i];
        __syncthreads();
    }
}

// ------------------------------------------------------------ trace and ||P||_F^2
// Block = red_rows(np) rows of one instance's P; partials (tr, ||.||^2) per block.
__global__ void __launch_bounds__(256) k_trace_frob_part(const Inst* __restrict__ insts,
                                                         const InstIO* __restrict__ io, Work we,
                                                         double* partials) {
    __shared__ double sh[33];
    const int i = find_inst(we.pre, 0, we.count, blockIdx.x);
    const int64_t n = insts[i].n, np = insts[i].np, ldp = io[i].ldp;
    const double* P = io[i].P;
    const int rows = red_rows(np);
    const int64_t r0 = (int64_t)(blockIdx.x - we.pre[i]) * rows;
    double tr = 0.0, fr = 0.0;
    if (insts[i].res->active) {
        for (int rr = 0; rr < rows; ++rr) {
            const int64_t r = r0 + rr;
            if (r >= n) break;
            const double* row = P + r * ldp;
            for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
                const double v = row[c];
                fr = fma(v, v, fr);
                if (c == r) tr += v;
            }
        }
    }
    tr = block_sum(tr, sh);
    fr = block_sum(fr, sh);
    if (threadIdx.x == 0) {
        partials[2 * (int64_t)blockIdx.x] = tr;
        partials[2 * (int64_t)blockIdx.x + 1] = fr;
    }
}

// One warp per instance: lane l sums partials l, l + 32, ... in order, then a fixed shuffle
// tree (deterministic for a given block count).
__global__ void k_trace_frob_final(const Inst* __restrict__ insts, Work we, const double* partials) {
    const int i = blockIdx.x;
    DevResult* r = insts[i].res;
    if (!r->active) return;
    double tr = 0.0, fr = 0.0;
    for (int b = we.pre[i] + (int)threadIdx.x; b < we.pre[i + 1]; b += 32) {
        tr += partials[2 * (int64_t)b];
        fr += partials[2 * (int64_t)b + 1];
    }
    tr = warp_sum(tr);
    fr = warp_sum(fr);
    if (threadIdx.x == 0) {
        r->trace = tr;
        r->frob2 = fr;
        r->trace_raw = tr;
        r->gamma = 0.0;
        r->proj = 0.0;
    }
}

// Trace of P from the partials of its float64-output product, one per 128 x 128 block on and
// above the diagonal; one block of 256 threads per instance, thread t sums blocks t, t + 256,
// ... in order, then a fixed shuffle and shared-memory tree (the same bits for every tile
// configuration of the product).
//  mode 0: tr P and ||P||_F^2 of the result (no correction).
//  mode 1: before the trace correction. The split products leave tr P off N_e by their
//    rounding (float32 masters: ~1e-8 N). The correction is the first-order shift of mu
//    that restores tr P = N_e: d f / d mu = f (1 - f) / kT for the Fermi function, so
//    P(mu + dmu) ~ P + gamma (P - P^2) with gamma = dmu / kT, and tr(P - P^2) = tr P -
//    ||P||_F^2 for symmetric P gives gamma = (N_e - tr P) / (tr P - ||P||_F^2). The
//    correction is a rounding correction, not a search for mu: it is applied only where it
//    moves P by less than the split forms' 1e-6 bar. With the eigenvalues of P in [0, 1],
//    ||P - P^2||_F <= sqrt(t) / 2 for t = tr(P - P^2), so ||gamma (P - P^2)||_F / sqrt(n) <=
//    |N_e - tr P| / (2 sqrt(t n)); where that bound exceeds 1e-6 (a learned mu accepted at a
//    loose trace tolerance), or |gamma| > 1/4, gamma = 0 and P keeps its trace. Every
//    instance without a failed stage is made active again (learned mu parks the accepted
//    ones) for the correcting product.
//  mode 2: after the correcting product, whose own split-product rounding leaves a float64
//    residual r = N_e - tr P (|gamma| times the rounding of tr P^2). The matrix nearest to P
//    in the Frobenius norm with trace N_e is P + (r / n) I: the block adds r / n to the n
//    diagonal entries when the correction was applied and |r| <= 1e-4 max(1, N_e) (a larger
//    residual is left in place for the caller to see) and sums the new diagonal for the
//    reported trace.
__global__ void k_tile_trace(const Inst* __restrict__ insts, const InstIO* __restrict__ io, const int* pre,
                             const double* part, int mode) {
    __shared__ double sh[33];
    const int i = blockIdx.x;
    DevResult* r = insts[i].res;
    if (mode == 1 ? r->status != FO_OK : !r->active) return;
    double tr = 0.0, fr = 0.0;
    for (int b = pre[i] + (int)threadIdx.x; b < pre[i + 1]; b += blockDim.x) {
        tr += part[2 * (int64_t)b];
        fr += part[2 * (int64_t)b + 1];
    }
    tr = block_sum(tr, sh);
    fr = block_sum(fr, sh);
    if (mode == 0) {
        if (threadIdx.x == 0) {
            r->trace = tr;
            r->frob2 = fr;
            r->trace_raw = tr;
            r->gamma = 0.0;
            r->proj = 0.0;
        }
        return;
    }
    const double n_e = io[i].n_e;
    if (mode == 1) {
        if (threadIdx.x == 0) {
            const double t = tr - fr;
            double g = (n_e - tr) / t;
            const double move = fabs(n_e - tr) / (2.0 * sqrt(t * (double)insts[i].n));
            const bool ok = t > 0.0 && isfinite(g) && fabs(g) <= 0.25 && move <= 1e-6;
            if (!ok) g = 0.0;
            r->trace_raw = tr;
            r->trace = tr;
            r->frob2 = fr;
            r->gamma = g;
            r->fixed = ok ? 1 : 0;
            r->proj = 0.0;
            r->active = 1;
        }
        return;
    }
    const int64_t n = insts[i].n, ldp = io[i].ldp;
    double* P = io[i].P;
    const double res = n_e - tr;
    double d = 0.0;
    if (r->fixed && fabs(res) <= 1e-4 * fmax(1.0, n_e) && isfinite(res)) d = res / (double)n;
    double t2 = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const double v = P[j * ldp + j] + d;
        if (d != 0.0) P[j * ldp + j] = v;
        t2 += v;
    }
    t2 = block_sum(t2, sh);
    if (threadIdx.x == 0) {
        // ||P + d I||^2 = ||P||^2 + 2 d tr P + n d^2
        r->frob2 = fr + 2.0 * d * tr + (double)n * d * d;
        r->trace = t2;
        r->proj = d;
    }
}

// P = R_0 (m = 1): slot n_tslots to the instance's float64 P.
__global__ void k_copy_out(const Inst* __restrict__ insts, const InstIO* __restrict__ io, Work we,
                           int slot, int is64) {
    const int i = find_inst(we.pre, 0, we.count, blockIdx.x);
    if (!insts[i].res->active) return;
    const int64_t n = insts[i].n, np = insts[i].np, ldp = io[i].ldp;
    const int rows = ew_rows(np);
    const int64_t r0 = (int64_t)(blockIdx.x - we.pre[i]) * rows;
    const char* src = insts[i].slots + insts[i].slot_bytes * slot;
    double* P = io[i].P;
    for (int rr = 0; rr < rows; ++rr) {
        const int64_t r = r0 + rr;
        if (r >= n) break;
        for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
            // float32 masters are kept on and above the diagonal only
            const int64_t q = is64 || c >= r ? r * np + c : c * np + r;
            P[r * ldp + c] = is64 ? reinterpret_cast<const double*>(src)[q]
                                  : (double)reinterpret_cast<const float*>(src)[q];
        }
    }
}

int grid_for(int64_t total, int threads) {
    int64_t b = (total + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

cudaError_t launch_set_io(const InstIO* ios, int count, InstIO* d_io, const Inst* d_inst, int first,
                          cudaStream_t s) {
    for (int c0 = 0; c0 < count; c0 += kIoChunk) {
        IoChunk p;
        p.count = count - c0 < kIoChunk ? count - c0 : kIoChunk;
        p.first = first + c0;
        for (int j = 0; j < p.count; ++j) p.io[j] = ios[c0 + j];
        k_set_io<<<1, kIoChunk, 0, s>>>(p, d_io, d_inst);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_bounds(const Inst* in, const InstIO* io, int batch, Work wg, double* part,
                          int use_given, cudaStream_t s) {
    if (use_given) {
        k_bounds_given<<<(batch + 127) / 128, 128, 0, s>>>(in, io, batch);
        return cudaGetLastError();
    }
    k_gershgorin_rows<<<wg.total, 32 * kGershRows, 0, s>>>(in, io, wg, part);
    k_gershgorin_final<<<batch, 256, 0, s>>>(in, wg, part);
    return cudaGetLastError();
}

cudaError_t launch_export_bounds(const DevResult* res, double* out3, cudaStream_t s) {
    k_export_bounds<<<1, 1, 0, s>>>(res, out3);
    return cudaGetLastError();
}

cudaError_t launch_scale(const Inst* in, const InstIO* io, Work ws, const Shape& sh, cudaStream_t s,
                         int* dbg) {
    k_scale_sym<<<ws.total, 256, 0, s>>>(in, io, ws, sh, dbg);
    return cudaGetLastError();
}

cudaError_t launch_pack_f32(const float* A, int64_t n, int64_t lda, char* slot, int64_t np, int planes,
                            int fp16, float pscale, cudaStream_t s) {
    k_pack_f32<<<grid_for(np * np, 256), 256, 0, s>>>(A, n, lda, slot, np, planes, fp16, pscale);
    return cudaGetLastError();
}

cudaError_t launch_diag_sums(const Inst* in, int batch, int count, const Shape& sh, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    k_diag_sums<<<dim3(count, batch), 256, 0, s>>>(in, sh.is64);
    return cudaGetLastError();
}

int gram_blocks_for(int64_t np, int is64) {
    const int64_t u = upper_chunks(np, kChunkBytes / (is64 ? 8 : 4));
    return (int)((u + kGChunks - 1) / kGChunks);
}

template <int TG, int TB, int TPW>
cudaError_t launch_gram_shape(const Inst* in, int batch, Work wgr, int giant0, int ngiant, int baby0, int nbaby,
                              int out_g0, int is64, cudaStream_t s, int* launches) {
    const int max_tiles = (kGramThreads / 32) * TPW;
    const int nbq = (nbaby + TB - 1) / TB;
    // giants per launch: the tiles fit the warps, and the staged rows stay <= kMaxRows
    int gmax = TG * (max_tiles / nbq);
    if (gmax > TG * ((kMaxRows - TB * nbq) / TG)) gmax = TG * ((kMaxRows - TB * nbq) / TG);
    if (gmax < TG) return cudaErrorInvalidValue;
    for (int g = 0; g < ngiant; g += gmax) {
        const int ng = ngiant - g < gmax ? ngiant - g : gmax;
        const int ngq = (ng + TG - 1) / TG;
        const size_t elem = is64 ? 8 : 4;
        const size_t smem = (size_t)kGStages * kCPS * (TG * ngq + TB * nbq) * (kChunkBytes / elem + 16 / elem) * elem;
        const int threads = gram_threads(ngq * nbq, TPW);
        if (is64) {
            cudaFuncSetAttribute(k_gram<double, TG, TB, TPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_gram<double, TG, TB, TPW><<<wgr.total, threads, smem, s>>>(in, wgr, giant0 + g, ng, baby0, nbaby);
        } else {
            cudaFuncSetAttribute(k_gram<float, TG, TB, TPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_gram<float, TG, TB, TPW><<<wgr.total, threads, smem, s>>>(in, wgr, giant0 + g, ng, baby0, nbaby);
        }
        const int npairs = ng * nbaby;
        k_sum_partials<<<dim3(npairs, batch), 128, 0, s>>>(in, npairs, (out_g0 + g) * nbaby);
        if (launches) *launches += 2;
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Tile shape of the Frobenius products for ngiant x nbaby pairs: 0 = two 4 x 4 tiles per warp
// (any size, several launches if needed); 1, 2, 3 = one 5 x 5, 4 x 5 or 5 x 4 tile per warp,
// taken when all pairs fit one launch of at most 16 warps. Among those the fewest staged-row
// reads per vector (tiles x (TG + TB)) wins, ties to the smaller tile.
int gram_shape(int ngiant, int nbaby) {
    const int shapes[4][3] = {{4, 4, 2}, {5, 5, 1}, {4, 5, 1}, {5, 4, 1}};
    int best = 0;
    long cost = 0;
    for (int i = 0; i < 4; ++i) {
        const int tg = shapes[i][0], tb = shapes[i][1], tpw = shapes[i][2];
        const int ngq = (ngiant + tg - 1) / tg, nbq = (nbaby + tb - 1) / tb;
        const bool fits = ngq * nbq <= (kGramThreads / 32) * tpw && tg * ngq + tb * nbq <= kMaxRows;
        if (i > 0 && !fits) continue;
        const long c = (long)ngq * nbq * (tg + tb);
        if (i == 0 || c < cost) {
            best = i;
            cost = c;
        }
    }
    return best;
}

// Register tiles of the float32 ring kernel (TG giant x TB baby rows per warp).
constexpr int kRingShapes[][2] = {{10, 10}, {8, 10}, {8, 9}, {10, 8}, {8, 8}, {6, 10}, {4, 10}, {2, 10}};
constexpr int kNumRingShapes = (int)(sizeof(kRingShapes) / sizeof(kRingShapes[0]));

// Giant row groups one ring launch takes for a tile shape: the tiles fit the consumer warps
// and the staged rows fit the ring; 0 when the babies alone do not fit.
int ring_groups_per_launch(int tg, int tb, int ngiant, int nbaby) {
    const int ngq = (ngiant + tg - 1) / tg, nbq = (nbaby + tb - 1) / tb;
    int g = kRMaxCons / nbq;
    if (g > (kRMaxRows - tb * nbq) / tg) g = (kRMaxRows - tb * nbq) / tg;
    if (g > ngq) g = ngq;
    return g < 1 ? 0 : g;
}

// Tile shape of the ring kernel for ngiant x nbaby pairs: the fewest launches (each launch
// reads every baby matrix once more), then the fewest multiply slots (padding rows cost
// FMAs and shared reads), then the fewest staged rows. -1 when none fits.
int gram_ring_shape(int ngiant, int nbaby) {
    int best = -1;
    long bl = 0, bs = 0, br = 0;
    for (int i = 0; i < kNumRingShapes; ++i) {
        const int tg = kRingShapes[i][0], tb = kRingShapes[i][1];
        const int gp = ring_groups_per_launch(tg, tb, ngiant, nbaby);
        if (gp == 0) continue;
        const int ngq = (ngiant + tg - 1) / tg, nbq = (nbaby + tb - 1) / tb;
        const long l = (ngq + gp - 1) / gp, slots = (long)ngq * nbq * tg * tb, rows = (long)tg * ngq + tb * nbq;
        if (best < 0 || l < bl || (l == bl && (slots < bs || (slots == bs && rows < br)))) {
            best = i;
            bl = l;
            bs = slots;
            br = rows;
        }
    }
    return best;
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    }
    return n;
}

template <int TG, int TB>
cudaError_t launch_gram_ring(const Inst* in, int batch, Work wgr, const GramGeom& geom, int giant0, int ngiant,
                             int baby0, int nbaby, int out_g0, int* err, cudaStream_t s, int* launches) {
    const int gmax = TG * ring_groups_per_launch(TG, TB, ngiant, nbaby);
    if (gmax <= 0) return cudaErrorInvalidValue;
    const int nbq = (nbaby + TB - 1) / TB;
    for (int g = 0; g < ngiant; g += gmax) {
        const int ng = ngiant - g < gmax ? ngiant - g : gmax;
        const int ngq = (ng + TG - 1) / TG, tiles = ngq * nbq;
        const int H = tiles == 1 ? 8 : (tiles == 2 ? 4 : (tiles <= 4 ? 2 : 1));
        const int ncons = tiles * H;
        const int rows = TG * ngq + TB * nbq;
        // chunks per stage: as many as leave a ring of two stages in the budget
        int CPS = kRMaxCPS;
        while (CPS > 1 && (int)(kRSmemBudget / ((size_t)rows * CPS * kChunkBytes)) < 2) --CPS;
        const size_t stage_bytes = (size_t)rows * CPS * kChunkBytes;
        int S = (int)(kRSmemBudget / stage_bytes);
        if (S > kRMaxStages) S = kRMaxStages;
        if (S < 2) return cudaErrorInvalidValue;
        const size_t smem = 1024 + (size_t)S * stage_bytes + 2 * kRMaxStages * sizeof(uint64_t) +
                            (size_t)ncons * 32 * 4 * sizeof(float);
        cudaFuncSetAttribute(k_gram_ring<TG, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        for (int q = 0; q < geom.ngroups; ++q) {
            const GramGroup& gr = geom.grp[q];
            GramMaps maps;
            std::memset(&maps, 0, sizeof(maps));
            for (int b = 0; b < gr.nb; ++b) {
                const GramBucket& bk = geom.bk[gr.b0 + b];
                if (!gram_make_map(&maps.g[b], bk, geom.nslots, ng, nullptr) ||
                    !gram_make_map(&maps.b[b], bk, geom.nslots, nbaby, nullptr))
                    return cudaErrorInvalidValue;
            }
            const int u0 = geom.pre_host[gr.i0], u1 = geom.pre_host[gr.i1];
            if (u1 <= u0) continue;
            const int grid = u1 - u0 < sm_count() ? u1 - u0 : sm_count();
            k_gram_ring<TG, TB><<<grid, 32 * (ncons + 1), smem, s>>>(maps, in, wgr, u0, u1, gr.b0, giant0 + g, ng,
                                                                     baby0, nbaby, H, S, CPS, err);
            if (launches) *launches += 1;
        }
        const int npairs = ng * nbaby;
        k_sum_partials<<<dim3(npairs, batch), 128, 0, s>>>(in, npairs, (out_g0 + g) * nbaby);
        if (launches) *launches += 1;
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_gram(const Inst* in, int batch, Work wgr, int giant0, int ngiant, int baby0, int nbaby,
                        int out_g0, int is64, const GramGeom* geom, int* err, cudaStream_t s, int* launches) {
    if (ngiant <= 0 || nbaby <= 0) return cudaSuccess;
    if (nbaby > 32) return cudaErrorInvalidValue;
    if (!is64 && geom) {
        switch (gram_ring_shape(ngiant, nbaby)) {
            case 0: return launch_gram_ring<10, 10>(in, batch, wgr, *geom, giant0, ngiant, baby0, nbaby, out_g0, err, s, launches);
            case 1: return launch_gram_ring<8, 10>(in, batch, wgr, *geom, giant0, ngiant, baby0, nbaby, out_g0, err, s, launches);
            case 2: return launch_gram_ring<8, 9>(in, batch, wgr, *geom, giant0, ngiant, baby0, nbaby, out_g0, err, s, launches);
            case 3: return launch_gram_ring<10, 8>(in, batch, wgr, *geom, giant0, ngiant, baby0, nbaby, out_g0, err, s, launches);
            case 4: return launch_gram_ring<8, 8>(in, batch, wgr, *geom, giant0, ngiant, baby0, nbaby, out_g0, err, s, launches);
            case 5: return launch_gram_ring<6, 10>(in, batch, wgr, *geom, giant0, ngiant, baby0, nbaby, out_g0, err, s, launches);
            case 6: return launch_gram_ring<4, 10>(in, batch, wgr, *geom, giant0, ngiant, baby0, nbaby, out_g0, err, s, launches);
            case 7: return launch_gram_ring<2, 10>(in, batch, wgr, *geom, giant0, ngiant, baby0, nbaby, out_g0, err, s, launches);
            default: break;   // no shape fits: the cp.async kernel below
        }
    }
    switch (gram_shape(ngiant, nbaby)) {
        case 1: return launch_gram_shape<5, 5, 1>(in, batch, wgr, giant0, ngiant, baby0, nbaby, out_g0, is64, s, launches);
        case 2: return launch_gram_shape<4, 5, 1>(in, batch, wgr, giant0, ngiant, baby0, nbaby, out_g0, is64, s, launches);
        case 3: return launch_gram_shape<5, 4, 1>(in, batch, wgr, giant0, ngiant, baby0, nbaby, out_g0, is64, s, launches);
        default: return launch_gram_shape<4, 4, 2>(in, batch, wgr, giant0, ngiant, baby0, nbaby, out_g0, is64, s, launches);
    }
}

cudaError_t launch_assemble_moments(const Inst* in, int batch, const Shape& sh, cudaStream_t s) {
    k_assemble_moments<<<batch, 64, 0, s>>>(in, sh.k, sh.m, sh.n_terms);
    return cudaGetLastError();
}

cudaError_t launch_tile_trace(const Inst* in, const InstIO* io, int batch, const int* pre, const double* part,
                              int mode, cudaStream_t s) {
    // 256 threads per instance: the partials and the diagonal of P (one sector per entry) are
    // read by enough threads to keep the loads in flight
    k_tile_trace<<<batch, 256, 0, s>>>(in, io, pre, part, mode);
    return cudaGetLastError();
}

cudaError_t launch_trace_frob(const Inst* in, const InstIO* io, Work we, double* part, cudaStream_t s) {
    k_trace_frob_part<<<we.total, 256, 0, s>>>(in, io, we, part);
    k_trace_frob_final<<<we.count, 32, 0, s>>>(in, we, part);
    return cudaGetLastError();
}

cudaError_t launch_copy_out(const Inst* in, const InstIO* io, Work we, const Shape& sh, cudaStream_t s) {
    k_copy_out<<<we.total, 256, 0, s>>>(in, io, we, sh.n_tslots, sh.is64);
    return cudaGetLastError();
}

}  // namespace fo
