// Split-precision recurrence product on the 5th-generation tensor cores (sm_103a).
//
//   out = alpha * sum_{(p,q) in products} A_p B_q^T + beta * C + D + shift * I_n
//
// A_p, B_q are the 16-bit planes of float32 working matrices (A = sum_p A_p), staged by
// TMA (cp.async.bulk.tensor, 64-byte swizzle) into a multi-stage shared-memory ring and
// multiplied by tcgen05.mma (kind::f16, M = 128, N = 256 or 128, K = 16) into float32
// accumulators in tensor memory. The epilogue applies the recurrence update (2 T_1 T_i -
// T_{i-1}, or 2 Y b_{l+1} - b_{l+2} + R_l for the Clenshaw giant steps) and writes the
// float32 master, the split planes of the result (the next product's operand) or the
// final float64 P.
//
// Grouped launch. One launch computes the same step for every instance of a batch: CTA b
// takes tile b of the concatenated tile lists (instances sorted by size, largest first, so
// the longest tiles start first). Operands are addressed through one 5-D tensor map per
// bucket of equally sized instances, (column, row, plane, slot, instance), passed as grid
// constants; the slot and the instance are TMA coordinates.
//
// Symmetric mode. Every matrix of the method is a polynomial in the symmetric X, so every
// product of two of them is symmetric. Only the tiles that hold an element on or above the
// diagonal are computed, and each such element is written twice, at (r, c) and (c, r); the
// stored matrices are then exactly symmetric, so reading B^T is exact, and about half of
// the tensor work is saved.
// (Reading B^T of a matrix that is only symmetric up to rounding makes the recurrence
// unstable: in the eigenbasis of X the pair (T_ab, T_ba) is multiplied by a matrix with
// eigenvalues +-2 sqrt(l_a l_b), which grows geometrically whenever l_a l_b < 0.)
//
// Plane storage (per plan). Full: every output tile is also written transposed, so each
// operand block is loaded K-major. Upper blocks: only the 128 x 128 blocks on and above the
// diagonal hold planes (the diagonal blocks whole); an operand block left of the diagonal
// is the transpose of a stored block and is loaded from it as an MN-major tile (boxes of 64
// columns x 32 rows, 128-byte swizzle), which saves the mirrored plane writes of the
// epilogue and about a quarter of the DRAM traffic but makes the tiles of the lower row
// blocks load more boxes. The autotuner picks whichever is faster for the batch (short
// tiles favour the upper blocks, long tiles the full storage); the products are the same
// sums in the same order, so the results are bit-identical.
//
// Accumulation. The tensor core rounds its float32 accumulator once per instruction, so a
// long chain of MMAs into one accumulator loses accuracy linearly in K. Each k-block (32 k)
// is therefore accumulated afresh into one of two TMEM accumulators (ping-pong) and drained
// by the epilogue warps into float32 registers while the next k-block accumulates into the
// other one. Within a k-block the correction products (a_0 b_1, a_1 b_0, ..., 2^-8 smaller)
// are issued first, while the accumulator is still small, and the leading product a_0 b_0
// last, so only two roundings per k-block happen at full magnitude.
//
// Tiles are 128 x TBN (TBN = 256 or 128, chosen per batch by the autotuner). With TBN = 256
// a column tile that reaches past the matrix edge by 128 columns runs as a 128-wide MMA and
// loads half the B rows; so does the diagonal tile of an odd 128-row block in symmetric mode,
// whose first 128 columns lie below the diagonal. A 256-wide tile moves half the B bytes per
// MMA cycle of a 128-wide one, which matters because the split forms load 2 to 6 operand
// planes per k-block.
//
// Roles (320 threads): warp 0 lane 0 issues TMA, warp 1 lane 0 issues MMAs (warp 1 owns the
// TMEM allocation), warps 2-9 drain TMEM: warp w reads lane quadrant (w & 3) = 32 tile rows
// and column half (w - 2) / 4. Every mbarrier wait is bounded by a %globaltimer deadline: on
// expiry the CTA raises a device error flag, drains what it has in flight (again bounded),
// frees its TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "fpbits.h"
#include "internal.cuh"

namespace fo {
namespace {

constexpr int kBM = 128;            // tile rows (UMMA M)
constexpr int kBK = 32;             // k elements per stage: 64 bytes of 16-bit data per row
constexpr int kRowBytes = kBK * 2;  // = swizzle span of CU_TENSOR_MAP_SWIZZLE_64B

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(c4)
        : "memory");
}
// Bulk prefetch of `bytes` (a multiple of 16) at a 16-byte aligned global address into L2.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<uint64_t>(p)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
// TMEM -> registers, 32 lanes x 32 columns; the wait is in the same asm block so that no
// use of the destination registers can be scheduled before the load has completed.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile with 64-byte swizzle: rows of
// 64 bytes, 8-row core groups 512 bytes apart (stride byte offset), descriptor version 1,
// layout type 4 = SWIZZLE_64B. The k16 slices inside the 64-byte row are addressed by
// advancing the start address (the swizzle is a function of the absolute address, and
// every stage buffer is 1024-byte aligned).
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;        // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)4 << 61;                 // SWIZZLE_64B
    return d;
}

// Shared-memory descriptor of an MN-major operand tile staged by TMA as boxes of 64 MN
// entries (128 bytes, 128-byte swizzle) x 32 k rows: 8-row core groups 1 KB apart along k
// (stride byte offset), 64-entry MN groups one 4 KB box apart (leading byte offset). The k16
// slices of a 32-wide k-block start 16 rows (2 KB) apart.
constexpr int kMnBoxCols = 64;
constexpr int kMnBoxBytes = kMnBoxCols * 2 * kBK;   // 4 KB
constexpr int kMnKStep = 16 * kMnBoxCols * 2;       // bytes per k16 slice
__device__ __forceinline__ uint64_t sdesc_mn128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(kMnBoxBytes >> 4) << 16;   // leading byte offset: next 64-entry MN group
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: next 8 k rows
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // SWIZZLE_128B
    return d;
}
constexpr uint32_t kIdescMnA = 1u << 15;   // instruction descriptor: A is MN-major
constexpr uint32_t kIdescMnB = 1u << 16;   // instruction descriptor: B is MN-major

// Instruction descriptor, kind::f16: float32 accumulator, A/B bf16 (1) or fp16 (0), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int tile_n, bool fp16) {
    return (1u << 4) | ((fp16 ? 0u : 1u) << 7) | ((fp16 ? 0u : 1u) << 10) |
           ((uint32_t)(tile_n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

constexpr int kBoxBytes = kBM * kRowBytes;   // one 128-row TMA box of one plane: 8 KB

struct TcMaps {
    CUtensorMap m[kMaxBuckets];    // boxes of 32 columns x 128 rows (K-major operand tiles)
    CUtensorMap mn[kMaxBuckets];   // boxes of 64 columns x 32 rows, 128-byte swizzle (MN-major tiles)
};

// MINB CTAs share an SM (1, or 2 for 128-wide tiles: one CTA's epilogue then overlaps the
// other's main loop); the shared-memory ring and the register budget are split accordingly.
// DW drain warps (8 or 16) read the TMEM accumulators: warp w serves lane quadrant w & 3 and
// column group (w - 2) / 4 of TBN / (DW / 4) columns; more drain warps keep more TMEM loads in
// flight per k-block.
template <int PA, int PB, int NPROD, bool F16, int TBN, int MINB, int DW>
struct TcCfg {
    static constexpr int kThreads = 32 * (2 + DW);
    static constexpr int kCols = TBN / (DW / 4);     // accumulator columns per drain warp
    static constexpr bool kLoad32 = MINB == 1 && DW == 8;   // else 16-column TMEM loads
    static constexpr int kBBoxes = TBN / kBM;
    static constexpr int kStageBytes = PA * kBoxBytes + PB * kBBoxes * kBoxBytes;
    static constexpr int kStagesRaw = (216 * 1024 / MINB) / kStageBytes;
    static constexpr int kStages = kStagesRaw > 8 ? 8 : (kStagesRaw < 2 ? 2 : kStagesRaw);
    static constexpr int kSmem = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
    static constexpr int kTmemCols = 2 * TBN;   // two accumulators (power of two >= 32)
    static_assert(kSmem <= 232448 - 64, "shared memory budget of one CTA exceeded");
    static_assert(MINB * kTmemCols <= 512, "tensor memory of the co-resident CTAs exceeded");
    static_assert(MINB * (kSmem + 1024) <= 233472, "shared memory of the co-resident CTAs exceeded");
    static constexpr int kRowPartOff = ((kBM * (TBN + 1) * 4 + 15) / 16) * 16;   // after the result tile
    static_assert(kStages * kStageBytes >= kRowPartOff + kBM * 2 * 2 * 8,
                  "result tile and trace partials must fit the stage ring");
};

// (a-plane, b-plane) of each product, largest first:
// (0,0) (0,1) (1,0) (0,2) (1,1) (2,0).
__host__ __device__ constexpr int prod_a(int p) { return p == 2 || p == 4 ? 1 : (p == 5 ? 2 : 0); }
__host__ __device__ constexpr int prod_b(int p) { return p == 1 || p == 4 ? 1 : (p == 3 ? 2 : 0); }

// Chain launches: bounded wait until *ctr >= need, with acquire semantics at GPU scope (the
// CTAs that counted released their stores). Gives up, returning false, when another CTA
// raised the device error flag or after the 2 s deadline.
__device__ bool wait_count(const int* ctr, int need, const int* err_flag) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= need) return true;
        if ((it & 63u) == 63u) {
            if (*reinterpret_cast<const volatile int*>(err_flag)) return false;
            const uint64_t t = gtimer();
            if (t0 == 0) t0 = t;
            else if (t - t0 > kWaitNs) return false;
        }
    }
}

// The 16-bit planes of two neighbouring entries, as the 32-bit words the stores write (low
// half: x0's plane, high half: x1's). BF16x3: p0 = bf16(x), p1 = bf16(x - p0), p2 =
// bf16(x - p0 - p1), each rounded to nearest; FP16x2: the entry scaled by pscale, p0 =
// fp16(x), p1 = fp16(x - p0). One packed conversion serves both entries of a plane.
__device__ __forceinline__ void split3x2(float x0, float x1, bool f16, float pscale, uint32_t& w0, uint32_t& w1,
                                         uint32_t& w2) {
    auto bits2 = [](auto v) {
        uint32_t u;
        memcpy(&u, &v, 4);
        return u;
    };
    if (!f16) {
        w0 = bits2(__floats2bfloat162_rn(x0, x1));
        const float r0 = x0 - __uint_as_float(w0 << 16), r1 = x1 - __uint_as_float(w0 & 0xffff0000u);
        w1 = bits2(__floats2bfloat162_rn(r0, r1));
        const float s0 = r0 - __uint_as_float(w1 << 16), s1 = r1 - __uint_as_float(w1 & 0xffff0000u);
        w2 = bits2(__floats2bfloat162_rn(s0, s1));
    } else {
        const float y0 = x0 * pscale, y1 = x1 * pscale;
        const __half2 f = __floats2half2_rn(y0, y1);
        const float2 b = __half22float2(f);
        w0 = bits2(f);
        w1 = bits2(__floats2half2_rn(y0 - b.x, y1 - b.y));
        w2 = 0;
    }
}

// Tile decode of one instance. Symmetric mode: the tiles of the 128-row block I that hold
// an element with col >= row, i.e. column tiles J >= (128 I) / TBN, enumerated row by row.
__device__ __forceinline__ void tile_of(int t, int tm, int tn, int tbn, int sym, int& I, int& J) {
    if (sym) {
        I = 0;
        int b = t;
        for (;;) {
            const int first = (I * kBM) / tbn;
            const int cnt = tn - first;
            if (b < cnt) { J = first + b; return; }
            b -= cnt;
            ++I;
        }
    }
    I = t / tn;
    J = t - I * tn;
}

// CHAIN: one launch runs a chain of dependent steps (ChainList): tiles are taken by ticket, a
// tile waits for its instance's previous step and signals its own completion.
template <int PA, int PB, int NPROD, bool F16, int TBN, int MINB, int DW, bool CHAIN>
__global__ void __launch_bounds__(32 * (2 + DW), MINB)
    k_tc_gemm(const __grid_constant__ TcMaps maps,
              const __grid_constant__ std::conditional_t<CHAIN, ChainList, StepList> steps,
              const Inst* __restrict__ insts, const InstIO* __restrict__ io, const int* __restrict__ pre,
              int i0, int i1, int tile0, int tiles, int b0, int sym, int* err_flag) {
    using Cfg = TcCfg<PA, PB, NPROD, F16, TBN, MINB, DW>;
    constexpr int S = Cfg::kStages;
    constexpr int NC = Cfg::kCols;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * Cfg::kStageBytes);
    uint64_t* empty = full + S;
    uint64_t* seg_full = empty + S;
    uint64_t* seg_empty = seg_full + 2;
    uint64_t* acc_full = seg_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);
    __shared__ int abort_flag;

    // ---------------- step, instance and tile of this CTA (uniform across the CTA)
    int sidx, gtile, inst;
    // chain launches: the ticket's step and the tile count its instance must reach first,
    // kept in shared memory (re-read after the main loop instead of held in registers)
    __shared__ int s_chain[4];   // ticket, step, count needed, stop
    if constexpr (CHAIN) {
        // the ticket decides the work: window, step within it, tile within the step. Whether
        // another CTA already gave up is read once, by thread 0, so that the whole CTA leaves
        // (or stays) together
        if (threadIdx.x == 0) {
            s_chain[0] = atomicAdd(steps.ticket, 1);
            s_chain[3] = *reinterpret_cast<const volatile int*>(err_flag);
        }
        __syncthreads();
        const int t = s_chain[0];
        int w = 0;
        while (w + 1 < steps.nwin && steps.win_base[w + 1] <= t) ++w;
        const int wi0 = steps.win_i0[w], wi1 = steps.win_i0[w + 1];
        const int w0 = __ldg(pre + wi0);
        const int tw = __ldg(pre + wi1) - w0;
        const int local = t - steps.win_base[w];
        sidx = local / tw;
        gtile = w0 + (local - sidx * tw);
        inst = find_inst(pre, wi0, wi1, gtile);
        if (s_chain[3]) return;   // a CTA gave up: the chain stops
        if (threadIdx.x == 0) {
            s_chain[1] = sidx;
            s_chain[2] = sidx * (__ldg(pre + inst + 1) - __ldg(pre + inst));
        }
    } else {
        sidx = (int)blockIdx.x / tiles;
        gtile = tile0 + (int)blockIdx.x - sidx * tiles;
        inst = find_inst(pre, i0, i1, gtile);
    }
    const Step& st = steps.s[sidx];
    const Inst& in = insts[inst];
    if (!step_needed(in.res, st.need_m)) {
        // an instance parked by the learned judge, or whose expansion does not need this
        // step: its tiles count as done
        if constexpr (CHAIN) {
            if (threadIdx.x == 0) atomicAdd(steps.done + (inst - i0), 1);
        }
        return;
    }
    const int np = (int)in.np;
    const CUtensorMap* map = &maps.m[in.bucket - b0];
    const CUtensorMap* map_mn = &maps.mn[in.bucket - b0];
    const bool ub = sym == 2;   // upper-block storage: lower operand blocks read transposed
    const int ib = in.in_bucket;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tm = np / kBM, tn = (np + TBN - 1) / TBN;
    int I, J;
    tile_of(gtile - __ldg(pre + inst), tm, tn, TBN, sym, I, J);
    const int m0 = I * kBM;
    int n0 = J * TBN;
    // k-blocks. The zero border past column n contributes exact zeros, so 128-wide tiles stop
    // at the k-block holding column n - 1 (short-K tiles of small matrices gain most); the
    // 256-wide kernels keep n_pad / 32, which they derive without another live register
    // (they run at their register cap, and the trimmed count made them spill)
    const int nk = TBN == 128 ? (int)((in.n + kBK - 1) / kBK) : np / kBK;
    // 128-row B boxes inside the matrix: a 256-wide tile at the edge may hold only one
    int nbox = (np - n0) / kBM < Cfg::kBBoxes ? (np - n0) / kBM : Cfg::kBBoxes;
    if (sym && n0 < m0) {
        // diagonal tile of an odd row block (256-wide tiles): its first 128 columns lie
        // below the diagonal, so only the 128 columns from the diagonal on are computed
        n0 = m0;
        nbox = 1;
    }
    const int tile_n = nbox * kBM;
    // columns the MMAs compute: up to the 32-column group holding column n - 1 (the zero border
    // past it contributes nothing; the epilogue writes the remaining columns as zeros), so the
    // edge tiles of a matrix whose n is not a multiple of the tile width issue narrower MMAs
    const int64_t nrem = in.n - n0;
    const int tile_k = nrem >= tile_n ? tile_n : (int)(((nrem + 31) / 32) * 32);
    const uint32_t idesc = idesc_f16(tile_k, F16);
    const uint32_t stage_tx = (uint32_t)(PA * kBoxBytes + PB * nbox * kBoxBytes);

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&seg_full[b], 1);
            mbar_init(&seg_empty[b], 32 * DW);
        }
        mbar_init(acc_full, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
        if (sym == 2) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map_mn)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(Cfg::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    volatile int* vabort = &abort_flag;

    auto stage_a = [&](int s, int p) { return smem + s * Cfg::kStageBytes + p * kBoxBytes; };
    auto stage_b = [&](int s, int p) {
        return smem + s * Cfg::kStageBytes + PA * kBoxBytes + p * Cfg::kBBoxes * kBoxBytes;
    };

    float2 sum[NC / 2];  // a drain thread's accumulated columns of its tile row, in pairs
#pragma unroll
    for (int j = 0; j < NC / 2; ++j) sum[j] = make_float2(0.0f, 0.0f);
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (instantiated per plane storage, as the MMA issuer)
            int issued = 0;
            if constexpr (CHAIN) {
                // the previous step's tiles of this instance (its stores are read by TMA, an
                // async-proxy read, after the generic-proxy acquire: the proxy fence orders them)
                const int need = *reinterpret_cast<volatile int*>(&s_chain[2]);
                if (need > 0 && !wait_count(steps.done + (inst - i0), need, err_flag)) {
                    atomicExch(&abort_flag, 1);
                    atomicExch(err_flag, 1);
                }
                asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            auto produce = [&](auto ub_tag) {
                constexpr bool U = decltype(ub_tag)::value;
                for (int kb = 0; kb < nk; ++kb) {
                    if (CHAIN && kb == 0 && *vabort) break;
                    const int s = kb % S;
                    if (kb >= S) {
                        if (!mbar_wait(&empty[s], ((kb / S) - 1) & 1, kWaitNs, vabort)) {
                            atomicExch(&abort_flag, 1);
                            atomicExch(err_flag, 1);
                            break;
                        }
                    }
                    if (!FO_CHK(st.dbg, kb * kBK < np && m0 + kBM <= np && n0 + tile_n <= np, 108, m0, n0)) {
                        atomicExch(&abort_flag, 1);
                        break;
                    }
                    mbar_expect_tx(&full[s], stage_tx);
                    // upper-block storage: a 128-row operand block left of the diagonal block is
                    // not stored; its transpose (above the diagonal) is loaded as an MN-major tile
                    const int KB = kb * kBK / kBM;
                    const bool a_mn = U && KB < m0 / kBM;
#pragma unroll
                    for (int p = 0; p < PA; ++p) {
                        if (!a_mn) {
                            tma_load_5d(stage_a(s, p), map, &full[s], kb * kBK, m0, p, st.a, ib);
                        } else {
#pragma unroll
                            for (int q = 0; q < kBM / kMnBoxCols; ++q)
                                tma_load_5d(stage_a(s, p) + q * kMnBoxBytes, map_mn, &full[s],
                                            m0 + kMnBoxCols * q, kb * kBK, p, st.a, ib);
                        }
                    }
#pragma unroll
                    for (int p = 0; p < PB; ++p)
                        for (int j = 0; j < nbox; ++j) {
                            if (!(U && KB < n0 / kBM + j)) {
                                tma_load_5d(stage_b(s, p) + j * kBoxBytes, map, &full[s], kb * kBK, n0 + j * kBM,
                                            p, st.b, ib);
                            } else {
#pragma unroll
                                for (int q = 0; q < kBM / kMnBoxCols; ++q)
                                    tma_load_5d(stage_b(s, p) + j * kBoxBytes + q * kMnBoxBytes, map_mn, &full[s],
                                                n0 + j * kBM + kMnBoxCols * q, kb * kBK, p, st.b, ib);
                            }
                        }
                    issued = kb + 1;
                }
            };
            if (ub) produce(std::true_type{});
            else produce(std::false_type{});
            // every operand is requested: bring the epilogue's C and D rows of this tile
            // into L2 while the last k-blocks are multiplied (prefetch hints, in bounds)
            if (!*vabort) {
                const char* sbase = insts[inst].slots;
                const int64_t sbytes = insts[inst].slot_bytes;
                const int cd[2] = {st.c, st.d};
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if (cd[q] < 0) continue;
                    const char* rows = sbase + sbytes * cd[q] + ((int64_t)m0 * np + n0) * 4;
                    for (int r = 0; r < kBM; ++r)
                        prefetch_l2(rows + (int64_t)r * np * 4, (uint32_t)tile_n * 4u);
                }
            }
            if (*vabort) {
                for (int kb = (issued > S ? issued - S : 0); kb < issued; ++kb)
                    mbar_wait(&full[kb % S], (kb / S) & 1, kDrainNs, nullptr);
            } else {
                // Producer tail: wait until the MMA warp has released every stage (the commit
                // arrivals of the last S k-blocks have landed) before the CTA may exit.
                for (int kb = (nk > S ? nk - S : 0); kb < nk; ++kb)
                    if (!mbar_wait(&empty[kb % S], (kb / S) & 1, kWaitNs, vabort)) {
                        atomicExch(err_flag, 1);
                        break;
                    }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer: one k-block per accumulator, corrections first.
            // The loop is instantiated once per plane storage, so the K-major one carries no
            // trace of the MN-major layouts (a runtime layout branch in it cost 5%).
            // Descriptors: the address field (bits 0-13, address / 16) of a stage's operand is
            // the ring base's plus a compile-time offset, so each MMA's descriptor is one add.
            const uint64_t d_k = sdesc_sw64(smem_u32(smem)), d_mn = sdesc_mn128(smem_u32(smem));
            auto issue = [&](auto ub_tag) {
                constexpr bool U = decltype(ub_tag)::value;
                for (int kb = 0; kb < nk; ++kb) {
                    const int s = kb % S, buf = kb & 1;
                    // operand layouts of this k-block (see the producer): K-major tiles advance
                    // 32 bytes per k16 slice, MN-major tiles 16 rows (2 KB)
                    const int KB = kb * kBK / kBM;
                    const bool a_mn = U && KB < m0 / kBM;
                    const bool b0_mn = U && KB < n0 / kBM;
                    const bool b1_mn = U && KB < n0 / kBM + 1;
                    const uint64_t so = (uint64_t)s * (uint64_t)(Cfg::kStageBytes >> 4);
                    auto adesc = [&](int p, int kk) {
                        return a_mn ? d_mn + so + (uint64_t)((p * kBoxBytes + kk * kMnKStep) >> 4)
                                    : d_k + so + (uint64_t)((p * kBoxBytes + kk * 32) >> 4);
                    };
                    auto bdesc = [&](int p, int kk, int j, bool mn) {
                        const int off = PA * kBoxBytes + (p * Cfg::kBBoxes + j) * kBoxBytes;
                        return mn ? d_mn + so + (uint64_t)((off + kk * kMnKStep) >> 4)
                                  : d_k + so + (uint64_t)((off + kk * 32) >> 4);
                    };
                    if (kb >= 2) {
                        if (!mbar_wait(&seg_empty[buf], ((kb >> 1) - 1) & 1, kWaitNs, vabort)) {
                            atomicExch(&abort_flag, 1);
                            atomicExch(err_flag, 1);
                            break;
                        }
                    }
                    if (!mbar_wait(&full[s], (kb / S) & 1, kWaitNs, vabort)) {
                        atomicExch(&abort_flag, 1);
                        atomicExch(err_flag, 1);
                        break;
                    }
                    fence_after();
                    const uint32_t d = tmem + buf * TBN;
                    // the two 128-column halves of B may differ in layout (the k-block of the
                    // diagonal block of the first half): one MMA per half when they do
                    const int halves = (!U || nbox == 1 || tile_k <= kBM || b0_mn == b1_mn) ? 1 : 2;
                    for (int j = 0; j < halves; ++j) {
                        const bool mn = j ? b1_mn : b0_mn;
                        const uint32_t id = (halves == 1 ? idesc : idesc_f16(j ? tile_k - kBM : kBM, F16)) |
                                            (a_mn ? kIdescMnA : 0u) | (mn ? kIdescMnB : 0u);
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk) {
#pragma unroll
                            for (int pr = 1; pr < NPROD; ++pr)
                                umma_f16(d + j * kBM, adesc(prod_a(pr), kk), bdesc(prod_b(pr), kk, j, mn), id,
                                         !(kk == 0 && pr == 1));
                        }
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk)
                            umma_f16(d + j * kBM, adesc(0, kk), bdesc(0, kk, j, mn), id, (NPROD > 1) || kk > 0);
                    }
                    umma_commit(&empty[s]);
                    umma_commit(&seg_full[buf]);
                }
            };
            if (ub) issue(std::true_type{});
            else issue(std::false_type{});
            // arrives once every issued MMA has completed (also after an abort)
            umma_commit(acc_full);
        }
        __syncwarp();
    } else {
        // ---------------- drain warps: add every finished k-block to registers
        const int q = warp & 3, grp = (warp - 2) >> 2;
        const uint32_t t_row = tmem + ((uint32_t)(q * 32) << 16) + grp * NC;
        // columns of this warp that the MMAs write (a multiple of 32): the others are never
        // read, so their sums stay zero, the value of the zero border there
        const int wcols = tile_k - grp * NC < 0 ? 0 : (tile_k - grp * NC > NC ? NC : tile_k - grp * NC);
        for (int kb = 0; kb < nk; ++kb) {
            const int buf = kb & 1;
            if (!mbar_wait_warp(&seg_full[buf], (kb >> 1) & 1, kWaitNs, vabort)) {
                ok = false;
                break;
            }
            __syncwarp();
            fence_after();
            if (Cfg::kLoad32) {
#pragma unroll
                for (int cb = 0; cb < NC / 32; ++cb) {
                    if (cb * 32 >= wcols) break;
                    uint32_t r[32];
                    tmem_ld32(t_row + buf * TBN + cb * 32, r);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        sum[cb * 16 + j] = __fadd2_rn(
                            sum[cb * 16 + j], make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1])));
                }
            } else {
                // half the registers per thread: 16-column loads
#pragma unroll
                for (int cb = 0; cb < NC / 16; ++cb) {
                    if (cb * 16 >= wcols) break;
                    uint32_t r[16];
                    tmem_ld16(t_row + buf * TBN + cb * 16, r);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        sum[cb * 8 + j] = __fadd2_rn(
                            sum[cb * 8 + j], make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1])));
                }
            }
            fence_before();
            mbar_arrive(&seg_empty[buf]);
        }
        // every MMA has completed before TMEM is freed
        if (!mbar_wait_warp(acc_full, 0, kWaitNs, nullptr)) ok = false;
        __syncwarp();
        if (!ok && lane == 0) {
            atomicExch(&abort_flag, 1);
            atomicExch(err_flag, 1);
        }
    }
    // ---------------- TMEM is no longer needed: free it before any global store
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(Cfg::kTmemCols));
    }
    if (warp < 2 || *vabort) return;  // uniform across the drain warps

    // the step's record again for the epilogue (derived anew, not held through the main loop)
    {
    const Step& st = steps.s[CHAIN ? *reinterpret_cast<volatile int*>(&s_chain[1]) : (int)blockIdx.x / tiles];
    // ---------------- drain warps: update and store through shared memory. The stage ring
    // is idle (every TMA load was consumed, every MMA completed), so it holds the 128 x TBN
    // float32 result tile; all global traffic below is coalesced across the warp.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    constexpr int LD = TBN + 1;
    float* tile = reinterpret_cast<float*>(smem);
    {
        const int q = warp & 3, grp = (warp - 2) >> 2;
        const int rl = q * 32 + lane;
#pragma unroll
        for (int c = 0; c < NC / 2; ++c) {
            tile[rl * LD + grp * NC + 2 * c] = st.alpha * sum[c].x;
            tile[rl * LD + grp * NC + 2 * c + 1] = st.alpha * sum[c].y;
        }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * DW) : "memory");
    if constexpr (CHAIN) {
        // every drain thread acquires the previous step's stores itself before its generic
        // loads of C and D (satisfied already: the producer waited before the first TMA);
        // after the accumulators went to shared memory, so none of them is live here. A wait
        // that gives up raises the error flag and goes on (the drain warps must all reach
        // their named barriers)
        const int need = *reinterpret_cast<volatile int*>(&s_chain[2]);
        if (need > 0 && !wait_count(steps.done + (inst - i0), need, err_flag)) atomicExch(err_flag, 1);
    }

    // instance fields of the epilogue, read here so that they are not live in the main loop
    const int64_t n_real = insts[inst].n;
    char* const base = insts[inst].slots;
    const int64_t sb = insts[inst].slot_bytes;
    const int64_t ld = np;
    const int64_t pstride = (int64_t)np * np;
    float* out_x = st.out >= 0 ? reinterpret_cast<float*>(base + sb * st.out) : nullptr;
    uint16_t* out_p = st.out >= 0 ? reinterpret_cast<uint16_t*>(base + sb * st.out + 4 * pstride) : nullptr;
    const float* Cm = st.c >= 0 ? reinterpret_cast<const float*>(base + sb * st.c) : nullptr;
    const float* Dm = st.d >= 0 ? reinterpret_cast<const float*>(base + sb * st.d) : nullptr;
    double* out64 = st.out64 ? io[inst].P : nullptr;
    const int64_t ldo = io[inst].ldp;
    const bool fix = out64 && st.fix64;
    const double gam = fix ? insts[inst].res->gamma : 0.0;
    const int planes = st.planes;
    const int ew = warp - 2;  // 0..DW-1
    // Trace and Frobenius partials per (tile row, 128-column block): each (row, 64-column
    // piece) is reduced by a fixed shuffle tree over the lanes and the two pieces of a block
    // are added in column order, so the partials, and the sums over their rows, do not depend
    // on the tile width or on which warp handled the row (every tiling gives the same bits);
    // kept in the idle stage ring after the result tile
    double (*rowpart)[2][2] = reinterpret_cast<double (*)[2][2]>(smem + Cfg::kRowPartOff);
    const float gam_f = (float)gam;
    // the caller's float64 P at the pair (grow, gcol), (grow, gcol + 1), for the flagged entries
    auto store64 = [&](int64_t grow, int64_t gcol, double x0, double x1, bool e0, bool e1) {
        double* dst = out64 + grow * ldo + gcol;
        if (e0) dst[0] = x0;
        if (e1) dst[1] = x1;
    };
    // contributions of the flagged entries (on or above the diagonal) to the trace, in float64,
    // and to ||P||_F^2 (strictly above counts twice), from their float32 values y: that sum only
    // sets gamma's denominator tr P - ||P||^2 and the reported ||P||^2, far above float32's
    // resolution (float64 arithmetic is the scarce pipe of this GPU)
    auto contrib = [&](int64_t grow, int64_t gcol, double x0, double x1, float y0, float y1, bool e0, bool e1,
                       double& ta, float& fa) {
        float f = 0.0f;
        if (e0) {
            if (gcol == grow) { ta += x0; f = fmaf(y0, y0, f); }
            else f = fmaf(2.0f * y0, y0, f);
        }
        if (e1) {
            if (gcol + 1 == grow) { ta += x1; f = fmaf(y1, y1, f); }
            else f = fmaf(2.0f * y1, y1, f);
        }
        fa = f;
    };
    // slot store (float32 master and 16-bit planes) of the same pair
    auto store_slot = [&](int64_t grow, int64_t gcol, float v0, float v1, bool w0, bool w1, bool master) {
        if (!(w0 || w1) || (!out_x && planes == 0)) return;
        const int64_t o = grow * ld + gcol;
        if (!FO_CHK(st.dbg, o >= 0 && o + 2 <= ld * ld, 111, grow, gcol)) return;
        uint32_t q0 = 0, q1 = 0, q2 = 0;   // the planes of the pair, one 32-bit word each
        if (planes > 0) split3x2(v0, v1, F16, st.plane_scale, q0, q1, q2);
        if (w0 && w1) {
            if (out_x && master) *reinterpret_cast<float2*>(out_x + o) = make_float2(v0, v1);
            if (planes > 0) {
                uint16_t* pl = out_p + o;
                *reinterpret_cast<uint32_t*>(pl) = q0;
                if (planes > 1) *reinterpret_cast<uint32_t*>(pl + pstride) = q1;
                if (planes > 2) *reinterpret_cast<uint32_t*>(pl + 2 * pstride) = q2;
            }
        } else {
            const int e = w0 ? 0 : 1;
            const float v = w0 ? v0 : v1;
            if (out_x && master) out_x[o + e] = v;
            if (planes > 0) {
                uint16_t* pl = out_p + o + e;
                const int sh = w0 ? 0 : 16;
                pl[0] = (uint16_t)(q0 >> sh);
                if (planes > 1) pl[pstride] = (uint16_t)(q1 >> sh);
                if (planes > 2) pl[2 * pstride] = (uint16_t)(q2 >> sh);
            }
        }
    };

    // The passes are instantiated twice: the products that write the caller's float64 P (with
    // their trace partials) and all others, whose loops then carry none of that code (a shared
    // loop with run-time checks made every product ~13 % slower).
    auto passes = [&](auto f64_tag) {
    constexpr bool F64 = decltype(f64_tag)::value;
    // row pass: each drain warp takes kBM / DW tile rows, lanes on column pairs; applies
    // beta C + D + shift and stores the entries with col >= row (all of them when not sym).
    // The C and D operands of G consecutive (row, column piece) iterations are loaded before
    // any of them is used, so that G loads per lane are in flight instead of one: C (two
    // products old) and D are DRAM reads, and one at a time they set the epilogue's pace.
    // (D may be the output slot itself, R_l -> b_l: each entry is read and then written by
    // the same thread, and the mirror pass below writes only entries that no row pass reads.)
    constexpr int RPW = kBM / DW;          // tile rows per drain warp
    constexpr int HPR = TBN / 64;          // 64-column pieces per row
    constexpr int NIT = RPW * HPR;
    constexpr int G = DW == 16 ? 4 : 8;    // 16 drain warps run at the 96-register cap
    static_assert(NIT % G == 0, "row-pass groups");
    for (int q0 = 0; q0 < NIT; q0 += G) {
        float2 cv[G], dv[G];
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const int q = q0 + u, rr = q / HPR, h = q % HPR;
            const int r = ew * RPW + rr, c = h * 64 + 2 * lane;
            const int64_t o = ((int64_t)m0 + r) * ld + n0 + c;
            cv[u] = make_float2(0.f, 0.f);
            dv[u] = make_float2(0.f, 0.f);
            if (c < tile_n) {
                // within a chain launch other SMs wrote C and D during this launch: L2 loads
                if (Cm) cv[u] = CHAIN ? __ldcg(reinterpret_cast<const float2*>(Cm + o))
                                      : *reinterpret_cast<const float2*>(Cm + o);
                if (Dm) dv[u] = CHAIN ? __ldcg(reinterpret_cast<const float2*>(Dm + o))
                                      : *reinterpret_cast<const float2*>(Dm + o);
            }
        }
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const int q = q0 + u, rr = q / HPR, h = q % HPR;
            const int r = ew * RPW + rr, c = h * 64 + 2 * lane;
            if (c >= tile_n) continue;   // past the matrix edge or the narrowed diagonal tile
            const int64_t grow = (int64_t)m0 + r, gcol = (int64_t)n0 + c;
            float v0 = tile[r * LD + c], v1 = tile[r * LD + c + 1];
            if (Cm) {
                v0 = fmaf(st.beta, cv[u].x, v0);
                v1 = fmaf(st.beta, cv[u].y, v1);
            }
            if (Dm) {
                v0 += dv[u].x;
                v1 += dv[u].y;
            }
            if (grow < n_real) {
                if (gcol == grow) v0 += st.shift;
                if (gcol + 1 == grow) v1 += st.shift;
            }
            tile[r * LD + c] = v0;
            tile[r * LD + c + 1] = v1;
            const bool w0 = !sym || gcol >= grow, w1 = !sym || gcol + 1 >= grow;
            double ta = 0.0;   // the diagonal entry, if this lane holds it
            float fa = 0.0f;
            if constexpr (F64) {
                const bool e0 = w0 && grow < n_real && gcol < n_real, e1 = w1 && grow < n_real && gcol + 1 < n_real;
                double x0 = widen_f32(v0), x1 = widen_f32(v1);
                float y0 = v0, y1 = v1;
                if (fix) {
                    // P is the float32 master C written by the last Clenshaw step (the float64 P it
                    // stands for is exactly its widening); the correction d = gamma (P - P P), ~1e-7
                    // of P, in float32, added in float64; the mirror pass adds the same d
                    const float d0 = gam_f * (cv[u].x - v0), d1 = gam_f * (cv[u].y - v1);
                    x0 = widen_f32(cv[u].x) + widen_f32(d0);
                    x1 = widen_f32(cv[u].y) + widen_f32(d1);
                    y0 = cv[u].x + d0;
                    y1 = cv[u].y + d1;
                    tile[r * LD + c] = d0;
                    tile[r * LD + c + 1] = d1;
                }
                if (out64) store64(grow, gcol, x0, x1, e0, e1);
                if (st.part) contrib(grow, gcol, x0, x1, y0, y1, e0, e1, ta, fa);
            }
            store_slot(grow, gcol, v0, v1, w0, w1, true);
            if (F64 && st.part) {
                // this (row, piece)'s sums (the `continue` above is uniform across the warp:
                // tile widths are multiples of 128); pieces 2b, 2b + 1 form the tile's
                // 128-column block b, added in that order by the warp that owns the row
                // ||P||^2: a float32 shuffle tree over the piece; the trace: the piece holds the
                // row's diagonal entry at most once, fetched from its lane (float64 work is
                // this GPU's scarcest: one shuffle instead of a float64 tree)
                for (int o = 16; o > 0; o >>= 1) fa += __shfl_xor_sync(0xffffffffu, fa, o);
                const int64_t dcol = grow - (gcol - 2 * lane);   // piece column of the diagonal
                double tv = 0.0;
                if (dcol >= 0 && dcol < 64) tv = __shfl_sync(0xffffffffu, ta, (int)(dcol >> 1));
                if (lane == 0) {
                    double* rp = rowpart[r][h >> 1];
                    if (h & 1) {
                        rp[0] += tv;
                        rp[1] += (double)fa;
                    } else {
                        rp[0] = tv;
                        rp[1] = (double)fa;
                    }
                }
            }
        }
    }
    if (F64 && st.part) {
        // the tile's 128 x 128 blocks: rows added in order; block (I, J) of the instance's
        // upper-block enumeration (row blocks in order, J >= I within a row)
        asm volatile("bar.sync 1, %0;" ::"n"(32 * DW) : "memory");
        const int nblk = tile_n / kBM;
        if (ew == 0 && lane < 2 * nblk) {
            const int b = lane >> 1, qty = lane & 1;
            double sacc = 0.0;
            for (int r = 0; r < kBM; ++r) sacc += rowpart[r][b][qty];
            const int64_t nb = np / kBM, I = m0 / kBM, J = n0 / kBM + b;
            const int64_t blk = (int64_t)st.part_pre[inst] + I * nb - I * (I - 1) / 2 + (J - I);
            st.part[2 * blk + qty] = sacc;
        }
    }
    if (!sym) return;
    // Below the diagonal the solver's slots need only the 16-bit planes (operands of later
    // products, read by TMA as whole rows); every float32 master read (epilogue C and D,
    // moments, contraction) stays on or above the diagonal.
    const bool lower_master = st.lower_master != 0;
    asm volatile("bar.sync 1, %0;" ::"n"(32 * DW) : "memory");
    // mirror pass: output row n0 + c holds tile column c for the entries with col > row;
    // each drain warp takes TBN / 8 tile columns, lanes on row pairs
    for (int cc = 0; cc < TBN / DW; ++cc) {
        const int c = ew * (TBN / DW) + cc;
        const int64_t grow = (int64_t)n0 + c;       // output row
        if (c >= tile_n) break;
        // upper-block storage keeps planes for the 128-row blocks on and above the diagonal
        // block only (a lower block is read as the transpose of its upper counterpart):
        // outside the tile's diagonal block nothing below the diagonal is written, except
        // into the caller's float64 P, which is returned whole
        const bool slot_rows = !(ub && !lower_master && grow >= (int64_t)m0 + kBM);
        if (!slot_rows && !(F64 && out64)) break;
#pragma unroll
        for (int h = 0; h < kBM / 64; ++h) {
            const int r = h * 64 + 2 * lane;
            const int64_t gcol = (int64_t)m0 + r;   // output column
            const float v0 = tile[r * LD + c], v1 = tile[(r + 1) * LD + c];
            if (F64 && out64) {
                // entries below the diagonal (counted twice by their mirrors above)
                const bool e0 = grow > gcol && grow < n_real && gcol < n_real;
                const bool e1 = grow > gcol + 1 && grow < n_real && gcol + 1 < n_real;
                if (fix) {
                    // the lower float32 master of P (written by the last Clenshaw step) + the d of the
                    // row pass: the bits of the mirrored entry
                    const float2 pm = *reinterpret_cast<const float2*>(Cm + grow * ld + gcol);
                    store64(grow, gcol, widen_f32(pm.x) + widen_f32(v0), widen_f32(pm.y) + widen_f32(v1), e0, e1);
                } else {
                    store64(grow, gcol, widen_f32(v0), widen_f32(v1), e0, e1);
                }
            }
            if (slot_rows) store_slot(grow, gcol, v0, v1, grow > gcol, grow > gcol + 1, lower_master);
        }
    }
    };
    if (out64 || st.part) passes(std::true_type{});
    else passes(std::false_type{});
    if constexpr (CHAIN) {
        // this tile's stores are complete: release them to the next step's tiles (generic
        // stores read later through TMA: a proxy fence as well), then count the tile
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __threadfence();
        asm volatile("bar.sync 1, %0;" ::"n"(32 * DW) : "memory");
        if (ew == 0 && lane == 0 && s_chain[0] != steps.drop) atomicAdd(steps.done + (inst - i0), 1);
    }
    }
}

// ------------------------------------------------------------------ persistent kernel
// One CTA per SM walks the launch's tiles (t = blockIdx.x, + gridDim.x, ...; the work list is
// ordered largest first, so every CTA gets a similar mix and the last tiles are the
// smallest). 128-wide tiles. Roles:
//   warp 0 lane 0   TMA producer, k-blocks of successive tiles into one ring;
//   warp 1 lane 0   MMA issuer into two TMEM accumulators (ping-pong per k-block);
//   DW drain warps  add every finished k-block to float32 registers; at the end of a tile
//                   they write alpha * sum into a result buffer in shared memory and move
//                   on to the next tile's k-blocks;
//   EW epilogue warps take the result buffer: the same row and mirror passes as k_tc_gemm
//                   (C, D, shift, plane split, mirrored stores, float64 P, trace
//                   partials), then hand the buffer back.
// So the epilogue of tile i runs while the MMAs of tile i + 1 do (the one-tile-per-CTA
// kernel leaves the tensor pipe idle during its epilogue), and barrier set-up, TMEM
// allocation and the first TMA latency are paid once per CTA instead of once per tile.
// Barrier phases follow the CTA's running counts of k-blocks and tiles. Every wait is
// bounded as in k_tc_gemm; a CTA that gives up raises the error flag, lets every role leave
// its loop, waits (bounded) for its copies in flight and frees its TMEM.
template <int PA, int PB, int NPROD, bool F16, int DW, int EW>
struct PcCfg {
    static constexpr int TBN = 128;
    static constexpr int kThreads = 32 * (2 + DW + EW);
    static constexpr int kCols = TBN / (DW / 4);   // accumulator columns per drain warp
    static constexpr int kStageBytes = PA * kBoxBytes + PB * kBoxBytes;
    static constexpr int kLD = TBN + 1;
    static constexpr int kTileBytes = kBM * kLD * 4;
    static constexpr int kRowPartBytes = kBM * 2 * 8;
    static constexpr int kBarBytes = 512;
    static constexpr int kFixed = kTileBytes + kRowPartBytes + kBarBytes + 1024 /*align*/;
    static constexpr int kStagesRaw = (232448 - 64 - kFixed) / kStageBytes;
    static constexpr int kStages = kStagesRaw > 8 ? 8 : kStagesRaw;
    static constexpr int kSmem = kStages * kStageBytes + kFixed;
    static constexpr int kTmemCols = 2 * TBN;
    static_assert(kStages >= 2, "persistent kernel: too few ring stages");
    static_assert(kSmem <= 232448 - 64, "persistent kernel: shared memory budget exceeded");
    static_assert(kBM % EW == 0 && (kBM / EW) * (TBN / 64) % 8 == 0, "epilogue warp split");
};

// The tile of work item t of a launch (steps x tiles), as every role of the persistent
// kernel derives it.
struct PTile {
    int sidx, inst, m0, n0, nk, tile_k;
    bool active;
};
__device__ __forceinline__ void persist_tile(int t, int tiles, int tile0, const int* __restrict__ pre, int i0,
                                             int i1, const Inst* __restrict__ insts, int sym, const StepList& steps,
                                             PTile& d) {
    d.sidx = t / tiles;
    const int gt = tile0 + t - d.sidx * tiles;
    d.inst = find_inst(pre, i0, i1, gt);
    const Inst& in = insts[d.inst];
    d.active = step_needed(in.res, steps.s[d.sidx].need_m);
    const int np = (int)in.np;
    int I, J;
    tile_of(gt - __ldg(pre + d.inst), np / kBM, np / kBM, kBM, sym, I, J);
    d.m0 = I * kBM;
    d.n0 = J * kBM;
    d.nk = (int)((in.n + kBK - 1) / kBK);
    const int64_t nrem = in.n - d.n0;
    d.tile_k = nrem >= kBM ? kBM : (int)(((nrem + 31) / 32) * 32);
}

// The epilogue of one 128 x 128 tile of the persistent kernel, run by its EW epilogue warps
// (named barrier 1) from the result buffer `tile` (alpha A B^T, leading dimension LD): the
// same row and mirror passes as k_tc_gemm -- beta C + D + shift, float32 master and 16-bit
// planes on and above the diagonal, planes (and, with lower_master, masters) of the mirrored
// half, the caller's float64 P (out64; with fix64 the trace correction), and the trace
// partials of a float64-output product.
template <bool F16, int EW, int TBN, int LD>
__device__ __forceinline__ void persist_epilogue(const Step& st, const Inst* __restrict__ insts,
                                                 const InstIO* __restrict__ io, int inst, int m0, int n0, int sym,
                                                 bool ub, float* tile, double (*rowpart)[2], int ew, int lane) {
    const Inst& in = insts[inst];
    const int64_t n_real = in.n;
    const int64_t np = in.np;
    char* const base = in.slots;
    const int64_t sb = in.slot_bytes;
    const int64_t ld = np;
    const int64_t pstride = np * np;
    float* out_x = st.out >= 0 ? reinterpret_cast<float*>(base + sb * st.out) : nullptr;
    uint16_t* out_p = st.out >= 0 ? reinterpret_cast<uint16_t*>(base + sb * st.out + 4 * pstride) : nullptr;
    const float* Cm = st.c >= 0 ? reinterpret_cast<const float*>(base + sb * st.c) : nullptr;
    const float* Dm = st.d >= 0 ? reinterpret_cast<const float*>(base + sb * st.d) : nullptr;
    double* out64 = st.out64 ? io[inst].P : nullptr;
    const int64_t ldo = io[inst].ldp;
    const bool fix = out64 && st.fix64;
    const double gam = fix ? in.res->gamma : 0.0;
    const int planes = st.planes;
    const float gam_f = (float)gam;
    auto store64 = [&](int64_t grow, int64_t gcol, double x0, double x1, bool e0, bool e1) {
        double* dst = out64 + grow * ldo + gcol;
        if (e0) dst[0] = x0;
        if (e1) dst[1] = x1;
    };
    // trace in float64, ||P||_F^2 from the float32 values (as in k_tc_gemm)
    auto contrib = [&](int64_t grow, int64_t gcol, double x0, double x1, float y0, float y1, bool e0, bool e1,
                       double& ta, float& fa) {
        float f = 0.0f;
        if (e0) {
            if (gcol == grow) { ta += x0; f = fmaf(y0, y0, f); }
            else f = fmaf(2.0f * y0, y0, f);
        }
        if (e1) {
            if (gcol + 1 == grow) { ta += x1; f = fmaf(y1, y1, f); }
            else f = fmaf(2.0f * y1, y1, f);
        }
        fa = f;
    };
    auto store_slot = [&](int64_t grow, int64_t gcol, float v0, float v1, bool w0, bool w1, bool master) {
        if (!(w0 || w1) || (!out_x && planes == 0)) return;
        const int64_t o = grow * ld + gcol;
        if (!FO_CHK(st.dbg, o >= 0 && o + 2 <= ld * ld, 111, grow, gcol)) return;
        uint32_t q0 = 0, q1 = 0, q2 = 0;   // the planes of the pair, one 32-bit word each
        if (planes > 0) split3x2(v0, v1, F16, st.plane_scale, q0, q1, q2);
        if (w0 && w1) {
            if (out_x && master) *reinterpret_cast<float2*>(out_x + o) = make_float2(v0, v1);
            if (planes > 0) {
                uint16_t* pl = out_p + o;
                *reinterpret_cast<uint32_t*>(pl) = q0;
                if (planes > 1) *reinterpret_cast<uint32_t*>(pl + pstride) = q1;
                if (planes > 2) *reinterpret_cast<uint32_t*>(pl + 2 * pstride) = q2;
            }
        } else {
            const int e = w0 ? 0 : 1;
            const float v = w0 ? v0 : v1;
            if (out_x && master) out_x[o + e] = v;
            if (planes > 0) {
                uint16_t* pl = out_p + o + e;
                const int sh = w0 ? 0 : 16;
                pl[0] = (uint16_t)(q0 >> sh);
                if (planes > 1) pl[pstride] = (uint16_t)(q1 >> sh);
                if (planes > 2) pl[2 * pstride] = (uint16_t)(q2 >> sh);
            }
        }
    };
    // instantiated for float64-output products and the others (see k_tc_gemm)
    auto passes = [&](auto f64_tag) {
        constexpr bool F64 = decltype(f64_tag)::value;
        constexpr int RPW = kBM / EW;
        constexpr int HPR = TBN / 64;
        constexpr int NIT = RPW * HPR;
        constexpr int G = 8;
        static_assert(NIT % G == 0, "row-pass groups");
        for (int q0 = 0; q0 < NIT; q0 += G) {
            float2 cv[G], dv[G];
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int q = q0 + u, rr = q / HPR, h = q % HPR;
                const int r = ew * RPW + rr, c = h * 64 + 2 * lane;
                const int64_t o = ((int64_t)m0 + r) * ld + n0 + c;
                cv[u] = Cm ? *reinterpret_cast<const float2*>(Cm + o) : make_float2(0.f, 0.f);
                dv[u] = Dm ? *reinterpret_cast<const float2*>(Dm + o) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int q = q0 + u, rr = q / HPR, h = q % HPR;
                const int r = ew * RPW + rr, c = h * 64 + 2 * lane;
                const int64_t grow = (int64_t)m0 + r, gcol = (int64_t)n0 + c;
                float v0 = tile[r * LD + c], v1 = tile[r * LD + c + 1];
                if (Cm) {
                    v0 = fmaf(st.beta, cv[u].x, v0);
                    v1 = fmaf(st.beta, cv[u].y, v1);
                }
                if (Dm) {
                    v0 += dv[u].x;
                    v1 += dv[u].y;
                }
                if (grow < n_real) {
                    if (gcol == grow) v0 += st.shift;
                    if (gcol + 1 == grow) v1 += st.shift;
                }
                tile[r * LD + c] = v0;
                tile[r * LD + c + 1] = v1;
                const bool w0 = !sym || gcol >= grow, w1 = !sym || gcol + 1 >= grow;
                double ta = 0.0;   // the diagonal entry, if this lane holds it
                float fa = 0.0f;
                if constexpr (F64) {
                    const bool e0 = w0 && grow < n_real && gcol < n_real, e1 = w1 && grow < n_real && gcol + 1 < n_real;
                    double x0 = widen_f32(v0), x1 = widen_f32(v1);
                    float y0 = v0, y1 = v1;
                    if (fix) {
                        // P is the float32 master C written by the last Clenshaw step (the float64 P it
                        // stands for is exactly its widening); the correction d = gamma (P - P P), ~1e-7
                        // of P, in float32, added in float64; the mirror pass adds the same d
                        const float d0 = gam_f * (cv[u].x - v0), d1 = gam_f * (cv[u].y - v1);
                        x0 = widen_f32(cv[u].x) + widen_f32(d0);
                        x1 = widen_f32(cv[u].y) + widen_f32(d1);
                        y0 = cv[u].x + d0;
                        y1 = cv[u].y + d1;
                        tile[r * LD + c] = d0;
                        tile[r * LD + c + 1] = d1;
                    }
                    if (out64) store64(grow, gcol, x0, x1, e0, e1);
                    if (st.part) contrib(grow, gcol, x0, x1, y0, y1, e0, e1, ta, fa);
                }
                store_slot(grow, gcol, v0, v1, w0, w1, true);
                if (F64 && st.part) {
                    // (row, 64-column piece) sums by a fixed shuffle tree; the two pieces of
                    // the row added in column order (the same bits as k_tc_gemm's partials)
                    for (int o = 16; o > 0; o >>= 1) fa += __shfl_xor_sync(0xffffffffu, fa, o);
                    const int64_t dcol = grow - (gcol - 2 * lane);
                    double tv = 0.0;
                    if (dcol >= 0 && dcol < 64) tv = __shfl_sync(0xffffffffu, ta, (int)(dcol >> 1));
                    if (lane == 0) {
                        if (h & 1) {
                            rowpart[r][0] += tv;
                            rowpart[r][1] += (double)fa;
                        } else {
                            rowpart[r][0] = tv;
                            rowpart[r][1] = (double)fa;
                        }
                    }
                }
            }
        }
        if (F64 && st.part) {
            asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");
            if (ew == 0 && lane < 2) {
                double sacc = 0.0;
                for (int r = 0; r < kBM; ++r) sacc += rowpart[r][lane];
                const int64_t nb = np / kBM, I = m0 / kBM, J = n0 / kBM;
                const int64_t blk = (int64_t)st.part_pre[inst] + I * nb - I * (I - 1) / 2 + (J - I);
                st.part[2 * blk + lane] = sacc;
            }
        }
        if (!sym) return;
        const bool lower_master = st.lower_master != 0;
        asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");
        // mirror pass: output row n0 + c holds tile column c for the entries with col > row
        for (int cc = 0; cc < TBN / EW; ++cc) {
            const int c = ew * (TBN / EW) + cc;
            const int64_t grow = (int64_t)n0 + c;
            const bool slot_rows = !(ub && !lower_master && grow >= (int64_t)m0 + kBM);
            if (!slot_rows && !(F64 && out64)) break;
#pragma unroll
            for (int hh = 0; hh < kBM / 64; ++hh) {
                const int r = hh * 64 + 2 * lane;
                const int64_t gcol = (int64_t)m0 + r;
                const float v0 = tile[r * LD + c], v1 = tile[(r + 1) * LD + c];
                if (F64 && out64) {
                    const bool e0 = grow > gcol && grow < n_real && gcol < n_real;
                    const bool e1 = grow > gcol + 1 && grow < n_real && gcol + 1 < n_real;
                    if (fix) {
                        const float2 pm = *reinterpret_cast<const float2*>(Cm + grow * ld + gcol);
                        store64(grow, gcol, widen_f32(pm.x) + widen_f32(v0), widen_f32(pm.y) + widen_f32(v1), e0, e1);
                    } else {
                        store64(grow, gcol, widen_f32(v0), widen_f32(v1), e0, e1);
                    }
                }
                if (slot_rows) store_slot(grow, gcol, v0, v1, grow > gcol, grow > gcol + 1, lower_master);
            }
        }
        // (the buffer goes back through res_empty, which counts every epilogue thread)
    };
    if (out64 || st.part) passes(std::true_type{});
    else passes(std::false_type{});
}

template <int PA, int PB, int NPROD, bool F16, int DW, int EW>
__global__ void __launch_bounds__(32 * (2 + DW + EW), 1)
    k_tc_persist(const __grid_constant__ TcMaps maps, const __grid_constant__ StepList steps,
                 const Inst* __restrict__ insts, const InstIO* __restrict__ io, const int* __restrict__ pre,
                 int i0, int i1, int tile0, int tiles, int b0, int sym, int* err_flag) {
    using Cfg = PcCfg<PA, PB, NPROD, F16, DW, EW>;
    constexpr int S = Cfg::kStages;
    constexpr int NC = Cfg::kCols;
    constexpr int TBN = Cfg::TBN;
    constexpr int LD = Cfg::kLD;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* tile = reinterpret_cast<float*>(smem + S * Cfg::kStageBytes);
    double (*rowpart)[2] = reinterpret_cast<double (*)[2]>(smem + S * Cfg::kStageBytes + Cfg::kTileBytes);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * Cfg::kStageBytes + Cfg::kTileBytes + Cfg::kRowPartBytes);
    uint64_t* empty = full + S;
    uint64_t* seg_full = empty + S;
    uint64_t* seg_empty = seg_full + 2;
    uint64_t* acc_full = seg_empty + 2;
    uint64_t* res_full = acc_full + 1;
    uint64_t* res_empty = res_full + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(res_empty + 1);
    __shared__ int abort_flag;
    __shared__ int s_go;   // the epilogue group's decision for its next tile
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int work = tiles * steps.count;
    const bool ub = sym == 2;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&seg_full[b], 1);
            mbar_init(&seg_empty[b], 32 * DW);
        }
        mbar_init(acc_full, 1);
        mbar_init(res_full, 32 * DW);
        mbar_init(res_empty, 32 * EW);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(Cfg::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    volatile int* vabort = &abort_flag;
    auto give_up = [&]() {
        atomicExch(&abort_flag, 1);
        atomicExch(err_flag, 1);
    };
    auto stage_a = [&](int s, int p) { return smem + s * Cfg::kStageBytes + p * kBoxBytes; };
    auto stage_b = [&](int s, int p) { return smem + s * Cfg::kStageBytes + PA * kBoxBytes + p * kBoxBytes; };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            uint32_t g = 0;   // k-blocks issued by this CTA
            auto produce = [&](auto ub_tag) {
                constexpr bool U = decltype(ub_tag)::value;
                for (int t = blockIdx.x; t < work; t += gridDim.x) {
                    PTile d;
                    persist_tile(t, tiles, tile0, pre, i0, i1, insts, sym, steps, d);
                    if (!d.active) continue;
                    const Step& st = steps.s[d.sidx];
                    const Inst& in = insts[d.inst];
                    const CUtensorMap* map = &maps.m[in.bucket - b0];
                    const CUtensorMap* map_mn = &maps.mn[in.bucket - b0];
                    const int ib = in.in_bucket;
                    for (int kb = 0; kb < d.nk; ++kb, ++g) {
                        const int s = (int)(g % S);
                        if (g >= (uint32_t)S && !mbar_wait(&empty[s], ((g / S) - 1) & 1, kWaitNs, vabort)) {
                            give_up();
                            return;
                        }
                        mbar_expect_tx(&full[s], (uint32_t)((PA + PB) * kBoxBytes));
                        const int KB = kb * kBK / kBM;
                        const bool a_mn = U && KB < d.m0 / kBM;
                        const bool b_mn = U && KB < d.n0 / kBM;
#pragma unroll
                        for (int p = 0; p < PA; ++p) {
                            if (!a_mn) {
                                tma_load_5d(stage_a(s, p), map, &full[s], kb * kBK, d.m0, p, st.a, ib);
                            } else {
#pragma unroll
                                for (int q = 0; q < kBM / kMnBoxCols; ++q)
                                    tma_load_5d(stage_a(s, p) + q * kMnBoxBytes, map_mn, &full[s],
                                                d.m0 + kMnBoxCols * q, kb * kBK, p, st.a, ib);
                            }
                        }
#pragma unroll
                        for (int p = 0; p < PB; ++p) {
                            if (!b_mn) {
                                tma_load_5d(stage_b(s, p), map, &full[s], kb * kBK, d.n0, p, st.b, ib);
                            } else {
#pragma unroll
                                for (int q = 0; q < kBM / kMnBoxCols; ++q)
                                    tma_load_5d(stage_b(s, p) + q * kMnBoxBytes, map_mn, &full[s],
                                                d.n0 + kMnBoxCols * q, kb * kBK, p, st.b, ib);
                            }
                        }
                    }
                    // the epilogue's C and D rows of this tile into L2 (hints, in bounds)
                    const int np = (int)in.np;
                    const int cd[2] = {st.c, st.d};
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        if (cd[q] < 0) continue;
                        const char* rows = in.slots + in.slot_bytes * cd[q] + ((int64_t)d.m0 * np + d.n0) * 4;
                        for (int r = 0; r < kBM; ++r) prefetch_l2(rows + (int64_t)r * np * 4, (uint32_t)TBN * 4u);
                    }
                }
            };
            if (ub) produce(std::true_type{});
            else produce(std::false_type{});
            // before the CTA may exit: normally the MMA warp's release (commit arrivals) of the
            // last S stages; after an abort at least the landing of the copies in flight
            const uint32_t k0 = g > (uint32_t)S ? g - S : 0;
            if (*vabort) {
                for (uint32_t k = k0; k < g; ++k) mbar_wait(&full[k % S], (k / S) & 1, kDrainNs, nullptr);
            } else {
                for (uint32_t k = k0; k < g; ++k)
                    if (!mbar_wait(&empty[k % S], (k / S) & 1, kWaitNs, vabort)) {
                        give_up();
                        break;
                    }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer: one k-block per accumulator, corrections first
            uint32_t g = 0, h = 0;   // k-blocks consumed, accumulator uses
            const uint64_t d_k = sdesc_sw64(smem_u32(smem)), d_mn = sdesc_mn128(smem_u32(smem));
            auto issue = [&](auto ub_tag) {
                constexpr bool U = decltype(ub_tag)::value;
                for (int t = blockIdx.x; t < work; t += gridDim.x) {
                    PTile d;
                    persist_tile(t, tiles, tile0, pre, i0, i1, insts, sym, steps, d);
                    if (!d.active) continue;
                    const uint32_t idesc0 = idesc_f16(d.tile_k, F16);
                    for (int kb = 0; kb < d.nk; ++kb, ++g, ++h) {
                        const int s = (int)(g % S), buf = (int)(h & 1);
                        const int KB = kb * kBK / kBM;
                        const bool a_mn = U && KB < d.m0 / kBM;
                        const bool b_mn = U && KB < d.n0 / kBM;
                        const uint64_t so = (uint64_t)s * (uint64_t)(Cfg::kStageBytes >> 4);
                        auto adesc = [&](int p, int kk) {
                            return a_mn ? d_mn + so + (uint64_t)((p * kBoxBytes + kk * kMnKStep) >> 4)
                                        : d_k + so + (uint64_t)((p * kBoxBytes + kk * 32) >> 4);
                        };
                        auto bdesc = [&](int p, int kk) {
                            const int off = PA * kBoxBytes + p * kBoxBytes;
                            return b_mn ? d_mn + so + (uint64_t)((off + kk * kMnKStep) >> 4)
                                        : d_k + so + (uint64_t)((off + kk * 32) >> 4);
                        };
                        if (h >= 2 && !mbar_wait(&seg_empty[buf], ((h >> 1) - 1) & 1, kWaitNs, vabort)) {
                            give_up();
                            return;
                        }
                        if (!mbar_wait(&full[s], (g / S) & 1, kWaitNs, vabort)) {
                            give_up();
                            return;
                        }
                        fence_after();
                        const uint32_t dt = tmem + (uint32_t)(buf * TBN);
                        const uint32_t id = idesc0 | (a_mn ? kIdescMnA : 0u) | (b_mn ? kIdescMnB : 0u);
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk) {
#pragma unroll
                            for (int pr = 1; pr < NPROD; ++pr)
                                umma_f16(dt, adesc(prod_a(pr), kk), bdesc(prod_b(pr), kk), id, !(kk == 0 && pr == 1));
                        }
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk)
                            umma_f16(dt, adesc(0, kk), bdesc(0, kk), id, (NPROD > 1) || kk > 0);
                        umma_commit(&empty[s]);
                        umma_commit(&seg_full[buf]);
                    }
                }
            };
            if (ub) issue(std::true_type{});
            else issue(std::false_type{});
            umma_commit(acc_full);   // every issued MMA has completed (also after an abort)
        }
        __syncwarp();
    } else if (warp < 2 + DW) {
        // ---------------- drain warps: k-blocks into registers, the tile into shared memory
        const int q = warp & 3, grp = (warp - 2) >> 2;
        const uint32_t t_row = tmem + ((uint32_t)(q * 32) << 16) + grp * NC;
        uint32_t h = 0, nt = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < work && ok; t += gridDim.x) {
            PTile d;
            persist_tile(t, tiles, tile0, pre, i0, i1, insts, sym, steps, d);
            if (!d.active) continue;
            float2 sum[NC / 2];   // accumulated columns, in pairs
#pragma unroll
            for (int j = 0; j < NC / 2; ++j) sum[j] = make_float2(0.0f, 0.0f);
            // columns the MMAs write (the others keep the border's zero)
            const int wcols = d.tile_k - grp * NC < 0 ? 0 : (d.tile_k - grp * NC > NC ? NC : d.tile_k - grp * NC);
            for (int kb = 0; kb < d.nk; ++kb, ++h) {
                const int buf = (int)(h & 1);
                if (!mbar_wait_warp(&seg_full[buf], (h >> 1) & 1, kWaitNs, vabort)) {
                    ok = false;
                    break;
                }
                __syncwarp();
                fence_after();
#pragma unroll
                for (int cb = 0; cb < NC / 16; ++cb) {
                    if (cb * 16 >= wcols) break;
                    uint32_t r[16];
                    tmem_ld16(t_row + buf * TBN + cb * 16, r);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        sum[cb * 8 + j] = __fadd2_rn(
                            sum[cb * 8 + j], make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1])));
                }
                fence_before();
                mbar_arrive(&seg_empty[buf]);
            }
            if (!ok) break;
            // the epilogue warps have released the result buffer of the previous tile
            if (nt > 0 && !mbar_wait_warp(res_empty, (nt - 1) & 1, kWaitNs, vabort)) {
                ok = false;
                break;
            }
            const float alpha = steps.s[d.sidx].alpha;
            const int rl = q * 32 + lane;
#pragma unroll
            for (int c = 0; c < NC / 2; ++c) {
                tile[rl * LD + grp * NC + 2 * c] = alpha * sum[c].x;
                tile[rl * LD + grp * NC + 2 * c + 1] = alpha * sum[c].y;
            }
            mbar_arrive(res_full);
            ++nt;
        }
        // every MMA has completed before TMEM is freed
        if (!mbar_wait_warp(acc_full, 0, kWaitNs, nullptr)) ok = false;
        __syncwarp();
        if (!ok && lane == 0) give_up();
    } else {
        // ---------------- epilogue warps
        const int ew = warp - 2 - DW;   // 0..EW-1
        uint32_t nt = 0;
        for (int t = blockIdx.x; t < work; t += gridDim.x) {
            PTile d;
            persist_tile(t, tiles, tile0, pre, i0, i1, insts, sym, steps, d);
            if (!d.active) continue;
            // the group decides together: after every warp's (bounded) wait, one thread samples
            // the abort flag (which any role may raise at any time) into s_go between two group
            // barriers, so that no warp can be left alone at the group's named barrier
            if (!mbar_wait_warp(res_full, nt & 1, kWaitNs, vabort) && lane == 0) give_up();
            asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");
            if (ew == 0 && lane == 0) s_go = *vabort ? 0 : 1;
            asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");
            if (!s_go) break;
            persist_epilogue<F16, EW, TBN, LD>(steps.s[d.sidx], insts, io, d.inst, d.m0, d.n0, sym, ub, tile,
                                               rowpart, ew, lane);
            mbar_arrive(res_empty);
            ++nt;
        }
    }
    // ---------------- every role is done: free TMEM
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(Cfg::kTmemCols));
    }
}

// ------------------------------------------------------------------ host side
using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

EncodeFn get_encode(std::string* err) {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    if (!fn && err) *err = "cuTensorMapEncodeTiled entry point not available";
    return fn;
}

template <int PA, int PB, int NPROD, bool F16, int TBN, int MINB, int DW, bool CHAIN, class SL>
cudaError_t launch_tc(const TcMaps& maps, const SL& st, unsigned grid, const Inst* in, const InstIO* io,
                      const int* pre, int i0, int i1, int tile0, int tiles, int b0, int sym, int* err_flag,
                      cudaStream_t s) {
    using Cfg = TcCfg<PA, PB, NPROD, F16, TBN, MINB, DW>;
    auto kern = k_tc_gemm<PA, PB, NPROD, F16, TBN, MINB, DW, CHAIN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
    if (e != cudaSuccess) return e;
    kern<<<grid, Cfg::kThreads, Cfg::kSmem, s>>>(maps, st, in, io, pre, i0, i1, tile0, tiles, b0, sym, err_flag);
    return cudaGetLastError();
}

template <int PA, int PB, int NPROD, bool F16, bool CHAIN, class SL>
cudaError_t dispatch_tbn(int tile_n, int ctas, int drain, const TcMaps& maps, const SL& st, unsigned grid,
                         const Inst* in, const InstIO* io, const int* pre, int i0, int i1, int tile0, int tiles,
                         int b0, int sym, int* err_flag, cudaStream_t s) {
    if (tile_n == 256)
        return drain == 16 ? launch_tc<PA, PB, NPROD, F16, 256, 1, 16, CHAIN>(maps, st, grid, in, io, pre, i0, i1,
                                                                               tile0, tiles, b0, sym, err_flag, s)
                           : launch_tc<PA, PB, NPROD, F16, 256, 1, 8, CHAIN>(maps, st, grid, in, io, pre, i0, i1,
                                                                              tile0, tiles, b0, sym, err_flag, s);
    if (ctas == 2)
        return launch_tc<PA, PB, NPROD, F16, 128, 2, 8, CHAIN>(maps, st, grid, in, io, pre, i0, i1, tile0, tiles, b0,
                                                               sym, err_flag, s);
    return launch_tc<PA, PB, NPROD, F16, 128, 1, 8, CHAIN>(maps, st, grid, in, io, pre, i0, i1, tile0, tiles, b0, sym,
                                                           err_flag, s);
}

// The persistent kernel: one CTA per SM (its shared memory admits no second one).
template <int PA, int PB, int NPROD, bool F16>
cudaError_t launch_persist(const TcMaps& maps, const StepList& st, const Inst* in, const InstIO* io, const int* pre,
                           int i0, int i1, int tile0, int tiles, int b0, int sym, int* err_flag, cudaStream_t s) {
    constexpr int DW = 8, EW = 4;
    using Cfg = PcCfg<PA, PB, NPROD, F16, DW, EW>;
    auto kern = k_tc_persist<PA, PB, NPROD, F16, DW, EW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int work = tiles * st.count;
    const unsigned grid = (unsigned)(work < sms ? work : sms);
    kern<<<grid, Cfg::kThreads, Cfg::kSmem, s>>>(maps, st, in, io, pre, i0, i1, tile0, tiles, b0, sym, err_flag);
    return cudaGetLastError();
}

template <bool CHAIN, class SL>
cudaError_t dispatch_prec(int prec, int tile_n, int ctas, int drain, const TcMaps& maps, const SL& st, unsigned grid,
                          const Inst* in, const InstIO* io, const int* pre, int i0, int i1, int tile0, int tiles,
                          int b0, int sym, int* err_flag, cudaStream_t s) {
    switch (prec) {
        case FO_PREC_BF16X3:
            return dispatch_tbn<3, 3, 6, false, CHAIN>(tile_n, ctas, drain, maps, st, grid, in, io, pre, i0, i1,
                                                       tile0, tiles, b0, sym, err_flag, s);
        case FO_PREC_FP16X2:
            return dispatch_tbn<2, 2, 3, true, CHAIN>(tile_n, ctas, drain, maps, st, grid, in, io, pre, i0, i1,
                                                      tile0, tiles, b0, sym, err_flag, s);
        case FO_PREC_BF16X1:
            return dispatch_tbn<1, 1, 1, false, CHAIN>(tile_n, ctas, drain, maps, st, grid, in, io, pre, i0, i1,
                                                       tile0, tiles, b0, sym, err_flag, s);
        default: return cudaErrorInvalidValue;
    }
}

bool tile_config_ok(int prec, int tile_n, int ctas, int drain) {
    return tc_planes(prec) != 0 && (tile_n == 128 || tile_n == 256) && (ctas == 1 || ctas == 2) &&
           !(ctas == 2 && tile_n != 128) && (drain == 8 || drain == 16) && !(drain == 16 && tile_n != 256);
}

void copy_maps(TcMaps& tm, const void* maps, int nb) {
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    for (int b = 0; b < nb; ++b) {
        std::memcpy(&tm.m[b], static_cast<const char*>(maps) + 256 * (size_t)b, sizeof(CUtensorMap));
        std::memcpy(&tm.mn[b], static_cast<const char*>(maps) + 256 * (size_t)b + 128, sizeof(CUtensorMap));
    }
}

}  // namespace

int tc_planes(int prec) {
    switch (prec) {
        case FO_PREC_BF16X3: return 3;
        case FO_PREC_FP16X2: return 2;
        case FO_PREC_BF16X1: return 1;
        default: return 0;
    }
}

int64_t tc_tiles(int64_t np, int tile_n) {
    const int64_t tm = np / kBM, tn = (np + tile_n - 1) / tile_n;
    int64_t c = 0;
    for (int64_t I = 0; I < tm; ++I) c += tn - (I * kBM) / tile_n;
    return c;
}

bool tc_make_map(void* map128, const void* planes0, int64_t np, int nplanes, int nslots, int count,
                 int64_t slot_bytes, int64_t inst_bytes, bool fp16, std::string* err, bool mn) {
    EncodeFn enc = get_encode(err);
    if (!enc) return false;
    cuuint64_t dims[5] = {(cuuint64_t)np, (cuuint64_t)np, (cuuint64_t)nplanes, (cuuint64_t)nslots,
                          (cuuint64_t)count};
    cuuint64_t strides[4] = {(cuuint64_t)np * 2, (cuuint64_t)np * np * 2, (cuuint64_t)slot_bytes,
                             (cuuint64_t)inst_bytes};
    cuuint32_t box[5] = {(cuuint32_t)(mn ? kMnBoxCols : kBK), (cuuint32_t)(mn ? kBK : kBM), 1, 1, 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(reinterpret_cast<CUtensorMap*>(map128),
                     fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5,
                     const_cast<void*>(planes0), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     mn ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        if (err) *err = "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
        return false;
    }
    return true;
}

bool gram_make_map(void* map128, const GramBucket& b, int nslots, int box_slots, std::string* err) {
    EncodeFn enc = get_encode(err);
    if (!enc) return false;
    cuuint64_t dims[4] = {(cuuint64_t)b.np, (cuuint64_t)b.np, (cuuint64_t)nslots, (cuuint64_t)b.count};
    cuuint64_t strides[3] = {(cuuint64_t)b.np * 4, (cuuint64_t)b.slot_bytes, (cuuint64_t)b.inst_bytes};
    cuuint32_t box[4] = {128, 1, (cuuint32_t)box_slots, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(reinterpret_cast<CUtensorMap*>(map128), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                     const_cast<char*>(b.master0), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        if (err) *err = "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
        return false;
    }
    return true;
}

cudaError_t tc_gemm(int prec, int tile_n, int ctas, int drain, const Step* steps, int nsteps, const Inst* in,
                    const InstIO* io, const int* pre, int i0, int i1, int tile0, int tiles, const void* maps, int b0,
                    int nb, int* err_flag, cudaStream_t s, std::string* err, int sym, int persist) {
    if (!tile_config_ok(prec, tile_n, ctas, drain) || nb < 1 || nb > kMaxBuckets || !err_flag || nsteps < 1 ||
        nsteps > kMaxSteps || (persist && tile_n != 128)) {
        if (err) *err = "tc_gemm: unsupported precision, tile or bucket count";
        return cudaErrorInvalidValue;
    }
    if (tiles <= 0) return cudaSuccess;
    TcMaps tm;
    copy_maps(tm, maps, nb);
    StepList st;
    for (int q = 0; q < nsteps; ++q) st.s[q] = steps[q];
    st.count = nsteps;
    if (persist) {
        switch (prec) {
            case FO_PREC_BF16X3:
                return launch_persist<3, 3, 6, false>(tm, st, in, io, pre, i0, i1, tile0, tiles, b0, sym, err_flag, s);
            case FO_PREC_FP16X2:
                return launch_persist<2, 2, 3, true>(tm, st, in, io, pre, i0, i1, tile0, tiles, b0, sym, err_flag, s);
            case FO_PREC_BF16X1:
                return launch_persist<1, 1, 1, false>(tm, st, in, io, pre, i0, i1, tile0, tiles, b0, sym, err_flag, s);
            default: return cudaErrorInvalidValue;
        }
    }
    return dispatch_prec<false>(prec, tile_n, ctas, drain, tm, st, (unsigned)(tiles * nsteps), in, io, pre, i0, i1,
                                tile0, tiles, b0, sym, err_flag, s);
}

cudaError_t tc_chain(int prec, int tile_n, int ctas, int drain, const Step* steps, int nsteps, const Inst* in,
                     const InstIO* io, const int* pre_dev, const int* pre_host, int i0, int i1, const void* maps,
                     int b0, int nb, int* err_flag, int* counters, int win_tiles, cudaStream_t s, std::string* err,
                     int sym) {
    if (!tile_config_ok(prec, tile_n, ctas, drain) || nb < 1 || nb > kMaxBuckets || !err_flag || !counters ||
        nsteps < 1 || nsteps > kMaxChain || sym == 0 || i1 <= i0) {
        if (err) *err = "tc_chain: unsupported precision, tile, bucket or step count";
        return cudaErrorInvalidValue;
    }
    const int total = pre_host[i1] - pre_host[i0];
    if (total <= 0) return cudaSuccess;
    // the chain's tickets: windows of consecutive instances holding at least win_tiles tiles
    // per step (the last window takes the rest), each window step-major
    thread_local ChainList cl;   // large (steps, windows): the launch copies it
    std::memset(&cl, 0, sizeof(cl));
    for (int q = 0; q < nsteps; ++q) cl.s[q] = steps[q];
    cl.count = nsteps;
    int nw = 0, base = 0, j = i0;
    while (j < i1) {
        int k = j + 1;
        if (win_tiles > 0)
            while (k < i1 && pre_host[k] - pre_host[j] < win_tiles) ++k;
        else
            k = i1;
        if (nw == kMaxWin - 1) k = i1;   // the window table is full: the rest in one window
        cl.win_base[nw] = base;
        cl.win_i0[nw] = j;
        base += nsteps * (pre_host[k] - pre_host[j]);
        ++nw;
        j = k;
    }
    cl.win_base[nw] = base;
    cl.win_i0[nw] = i1;
    cl.nwin = nw;
    cl.ticket = counters;
    cl.done = counters + 1;
    // FERMI_CHAIN_DROP_SIGNAL=t: the tile of ticket t does not count itself done, so the tiles
    // waiting on it run out their bounded wait (tests of the timeout path; no fault involved)
    const char* drop = getenv("FERMI_CHAIN_DROP_SIGNAL");
    cl.drop = drop ? atoi(drop) : -1;
    cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(int) * (size_t)(1 + i1 - i0), s);
    if (e != cudaSuccess) return e;
    TcMaps tm;
    copy_maps(tm, maps, nb);
    return dispatch_prec<true>(prec, tile_n, ctas, drain, tm, cl, (unsigned)base, in, io, pre_dev, i0, i1, 0, 0, b0,
                               sym, err_flag, s);
}

}  // namespace fo
