// Spectral bounds without any device allocation (fo_spectral_bounds_noalloc).
//
// Some callers cannot allocate device memory at the point where they need the bounds: code
// running inside a memory pool they do not own, a host thread that must not touch the
// allocator while another component holds it, or an embedding that forbids cudaMalloc after
// start-up. This entry point needs neither a context nor a workspace: its per-block partial
// results live in a fixed file-scope device array, and the caller provides H and the output.
//
// The array is shared by every call on a device and keeps the contents of the last call.
// Each call writes every partial it later reads, so nothing has to be cleared; calls whose
// kernels overlap on the GPU (different streams, or several host threads) race on it and
// must be serialised by the caller.
#include <cuda_runtime.h>

#include "exactsum.h"
#include "internal.cuh"

namespace fo {
namespace {

constexpr int kRowsPerBlock = 8;                       // one warp per row, 8 warps per block
constexpr int kMaxBlocks = FO_NOALLOC_MAX_N / kRowsPerBlock;

// Per-block (min_i lo_i, max_i hi_i, any non-finite) of the Gershgorin discs: 4096 x 32 B = 128 KiB.
struct Partial {
    double lo, hi;
    int bad, pad_;
    double pad2_;
};
static __device__ __align__(256) Partial g_scratch[kMaxBlocks];

__device__ __forceinline__ double wsum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block b handles rows [8b, 8b + 8): warp w sums |h_ij|, j != i, of row 8b + w exactly (the
// 128-bit fixed-point sums of csrc/exactsum.h, rounded to float64 once), so that the bounds
// are the same bits as those of the context entry point, whatever the order of the terms.
__global__ void __launch_bounds__(32 * kRowsPerBlock) k_bounds_rows_static(const double* __restrict__ H,
                                                                           int64_t n, int64_t ld,
                                                                           Partial* part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t row = (int64_t)blockIdx.x * kRowsPerBlock + warp;
    double lo = INFINITY, hi = -INFINITY;
    int bad = 0;
    if (row < n) {
        const unsigned long long* r = reinterpret_cast<const unsigned long long*>(H + row * ld);
        XAcc acc{0, 0, 0};
        double d = 0.0;
        for (int64_t j = lane; j < n; j += 32) {
            const uint64_t v = r[j];
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
        d = wsum(d);
        lo = d - s;
        hi = d + s;
    }
    bad = __any_sync(0xffffffffu, bad);
    __shared__ double slo[kRowsPerBlock], shi[kRowsPerBlock];
    __shared__ int sbad[kRowsPerBlock];
    if (lane == 0) { slo[warp] = lo; shi[warp] = hi; sbad[warp] = bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        lo = slo[0];
        hi = shi[0];
        bad = sbad[0];
        for (int w = 1; w < kRowsPerBlock; ++w) {
            lo = fmin(lo, slo[w]);
            hi = fmax(hi, shi[w]);
            bad |= sbad[w];
        }
        part[blockIdx.x].lo = lo;
        part[blockIdx.x].hi = hi;
        part[blockIdx.x].bad = bad;
    }
}

// One block reduces the partials and writes emin, emax and the non-finite flag.
__global__ void k_bounds_final_static(const Partial* part, int nparts, double* out3) {
    __shared__ double slo[32], shi[32];
    __shared__ int sbad[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double lo = INFINITY, hi = -INFINITY;
    int bad = 0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        lo = fmin(lo, part[i].lo);
        hi = fmax(hi, part[i].hi);
        bad |= part[i].bad;
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
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
        out3[0] = lo;
        out3[1] = hi;
        out3[2] = bad ? 1.0 : 0.0;
    }
}

// Device address of g_scratch on the current device. In host code the symbol itself is only
// a host-side stand-in and must never be passed to a kernel. The address is looked up on
// every call (cudaGetSymbolAddress is cheap and allocates nothing) rather than cached: after
// a device reset or a re-created primary context the module is loaded anew, possibly at
// another address, and a cached pointer would be stale.
cudaError_t scratch_address(Partial** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<Partial*>(p);
    return cudaSuccess;
}

}  // namespace
}  // namespace fo

extern "C" fo_status fo_spectral_bounds_noalloc(const double* dH, int64_t n, int64_t ld,
                                                double* d_bounds, void* stream) {
    using namespace fo;
    if (!dH || !d_bounds || n < 1 || ld < n) return FO_ERR_ARG;
    if (n > FO_NOALLOC_MAX_N) return FO_ERR_ARG;   // beyond the fixed scratch capacity
    Partial* part = nullptr;
    if (scratch_address(&part) != cudaSuccess) {
        cudaGetLastError();
        return FO_ERR_CUDA;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int nparts = (int)((n + kRowsPerBlock - 1) / kRowsPerBlock);
    k_bounds_rows_static<<<nparts, 32 * kRowsPerBlock, 0, st>>>(dH, n, ld, part);
    k_bounds_final_static<<<1, 256, 0, st>>>(part, nparts, d_bounds);
    return cudaGetLastError() == cudaSuccess ? FO_OK : FO_ERR_CUDA;
}
