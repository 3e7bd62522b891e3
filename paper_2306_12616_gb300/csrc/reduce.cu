// Bandwidth-bound kernels of the solver: spectral bounds, scaling and plane splitting,
// traces, Frobenius inner products (moments) and the output copy.
//
// All reductions are deterministic: fixed per-thread order, warp shuffles, a fixed tree in
// shared memory, and per-block partials summed in block order by a final kernel.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

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

// ------------------------------------------------------------------ Gershgorin bounds
// One warp per row: r_i = sum_{j != i} |h_ij| (float64, lane-strided, shuffle tree),
// lo_i = h_ii - r_i, hi_i = h_ii + r_i; per-block min/max to partials.
__global__ void __launch_bounds__(256) k_gershgorin_rows(const double* __restrict__ H, int64_t n,
                                                         int64_t ld, double* part_lo,
                                                         double* part_hi, int* part_bad) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double lo = INFINITY, hi = -INFINITY;
    int bad = 0;
    for (int64_t row = (int64_t)blockIdx.x * nw + warp; row < n; row += (int64_t)gridDim.x * nw) {
        const double* r = H + row * ld;
        double s = 0.0, d = 0.0;
        for (int64_t j = lane; j < n; j += 32) {
            const double v = __ldg(r + j);
            bad |= !isfinite(v);
            if (j == row) d = v; else s += fabs(v);
        }
        s = warp_sum(s);
        d = warp_sum(d);
        lo = fmin(lo, d - s);
        hi = fmax(hi, d + s);
    }
    __shared__ double slo[32], shi[32];
    __shared__ int sbad[32];
    lo = warp_min(lo);
    hi = warp_max(hi);
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) { slo[warp] = lo; shi[warp] = hi; sbad[warp] = bad; }
    __syncthreads();
    if (warp == 0) {
        lo = lane < nw ? slo[lane] : INFINITY;
        hi = lane < nw ? shi[lane] : -INFINITY;
        bad = lane < nw ? sbad[lane] : 0;
        lo = warp_min(lo);
        hi = warp_max(hi);
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            part_lo[blockIdx.x] = lo;
            part_hi[blockIdx.x] = hi;
            part_bad[blockIdx.x] = bad;
        }
    }
}

__global__ void k_gershgorin_final(const double* part_lo, const double* part_hi,
                                   const int* part_bad, int nparts, DevResult* res) {
    __shared__ double slo[32], shi[32];
    __shared__ int sbad[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double lo = INFINITY, hi = -INFINITY;
    int bad = 0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        lo = fmin(lo, part_lo[i]);
        hi = fmax(hi, part_hi[i]);
        bad |= part_bad[i];
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
        res->bounds[0] = lo;
        res->bounds[1] = hi;
        res->nonfinite = bad;
        res->status = bad ? FO_ERR_NONFINITE : FO_OK;
    }
}

__global__ void k_set_scalar(double* dst, double v) { *dst = v; }

__global__ void k_export_bounds(const DevResult* res, double* out3) {
    out3[0] = res->bounds[0];
    out3[1] = res->bounds[1];
    out3[2] = res->nonfinite ? 1.0 : 0.0;
}

__global__ void k_set_bounds(DevResult* res, double emin, double emax) {
    res->bounds[0] = emin;
    res->bounds[1] = emax;
    res->nonfinite = 0;
    res->status = FO_OK;
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

// X = (2H - (emin+emax) I) / (emax - emin) into an np x np matrix with zero border, built
// from the upper triangle of H only, so that X is exactly symmetric. One block per 32 x 32
// tile (bi, bj), bj >= bi: the H tile is staged in shared memory and written to X at
// (bi, bj) and, transposed, at (bj, bi). Output float64, or float32 master + split planes.
template <bool F64>
__global__ void __launch_bounds__(256) k_scale_sym(const double* __restrict__ H, int64_t n,
                                                   int64_t ld, const DevResult* res,
                                                   double* __restrict__ X64, MatF32 X32,
                                                   int64_t np, int planes, int fp16,
                                                   float pscale, int* dbg) {
    __shared__ double tile[32][33];
    const int tn = (int)(np / 32);
    int bi = 0, b = blockIdx.x;
    while (b >= tn - bi) { b -= tn - bi; ++bi; }
    const int bj = bi + b;
    const double ea = res->bounds[0], eb = res->bounds[1];
    const double inv = 1.0 / (eb - ea), csum = ea + eb;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int ry = ty; ry < 32; ry += 8) {
        const int64_t r = (int64_t)bi * 32 + ry, c = (int64_t)bj * 32 + tx;
        tile[ry][tx] = (r < n && c < n) ? H[r * ld + c] : 0.0;
    }
    __syncthreads();
    for (int ry = ty; ry < 32; ry += 8) {
        // (bi*32 + ry, bj*32 + tx); in a diagonal tile the lower half mirrors the upper
        for (int pass = 0; pass < (bi == bj ? 1 : 2); ++pass) {
            int64_t r, c;
            double h;
            if (pass == 0) {
                r = (int64_t)bi * 32 + ry;
                c = (int64_t)bj * 32 + tx;
                h = (bi == bj && tx < ry) ? tile[tx][ry] : tile[ry][tx];
            } else {
                r = (int64_t)bj * 32 + ry;
                c = (int64_t)bi * 32 + tx;
                h = tile[tx][ry];
            }
            double v = 0.0;
            if (r < n && c < n) {
                v = 2.0 * h;
                if (r == c) v -= csum;
                v *= inv;
            }
            const int64_t idx = r * np + c;
            if (!FO_CHK(dbg, r < np && c < np, 201, r, c)) continue;
            if (F64) X64[idx] = v;
            else store_split((float)v, X32.x + idx, X32.planes + idx, X32.plane_stride, planes, fp16, pscale);
        }
    }
}

__global__ void k_pack_f32(const float* __restrict__ A, int64_t n, int64_t lda, MatF32 X,
                           int64_t np, int planes, int fp16, float pscale) {
    const int64_t total = np * np;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / np, col = idx - r * np;
        const float v = (r < n && col < n) ? A[r * lda + col] : 0.0f;
        store_split(v, X.x + idx, X.planes + idx, X.plane_stride, planes, fp16, pscale);
    }
}

// ----------------------------------------------------------------------- traces
// out[s] = sum_{i<n} slot_s[i, i] (float64), one block per slot.
__global__ void k_diag_sums(const char* base, int64_t slot_stride_bytes, int64_t n, int64_t np,
                            int is_f64, double* out) {
    __shared__ double sh[33];
    const char* slot = base + slot_stride_bytes * blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        s += is_f64 ? reinterpret_cast<const double*>(slot)[i * np + i]
                    : (double)reinterpret_cast<const float*>(slot)[i * np + i];
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// --------------------------------------------------------- Frobenius inner products
// gram[g * nbaby + b] = <S_{giant0+g}, S_{baby0+b}>_F over all np*np entries (the zero
// border contributes nothing). A block stages kChunk consecutive entries of every matrix in
// shared memory, matrix-major (row s holds the chunk of matrix s), with float4 loads. Each
// warp owns up to kTPW 4 x 4 tiles of (giant, baby) pairs; its lanes walk consecutive
// entries of a row, so shared-memory reads are conflict free. Within a chunk the products
// are summed in T; across chunks float32 sums are compensated (Kahan), float64 sums are
// plain. Lanes are reduced by shuffles at the end into per-block float64 partials.
constexpr int kChunk = 256;
constexpr int kRowPad = 4;
constexpr int kTPW = 2;

template <typename T>
__global__ void __launch_bounds__(512) k_gram(const char* base, int64_t slot_stride_bytes,
                                               int giant0, int ngiant, int baby0, int nbaby,
                                               int64_t total, double* partials) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    constexpr int RS = kChunk + kRowPad;                 // row stride (elements)
    const int ng4 = (ngiant + 3) / 4, nb4 = (nbaby + 3) / 4;
    const int nrows = 4 * (ng4 + nb4);
    const int ntiles = ng4 * nb4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    T acc[kTPW][16];
    T cmp[kTPW][16];   // Kahan compensation (float32 only)
#pragma unroll
    for (int t = 0; t < kTPW; ++t)
#pragma unroll
        for (int q = 0; q < 16; ++q) { acc[t][q] = T(0); cmp[t][q] = T(0); }

    constexpr int V = 16 / sizeof(T);                    // elements per 16-byte load
    const int64_t nchunks = (total + kChunk - 1) / kChunk;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t e0 = ch * kChunk;
        for (int q = threadIdx.x; q < nrows * (kChunk / V); q += blockDim.x) {
            const int srow = q / (kChunk / V), ev = (q % (kChunk / V)) * V;
            int slot = -1;
            if (srow < 4 * ng4) { if (srow < ngiant) slot = giant0 + srow; }
            else { const int bb = srow - 4 * ng4; if (bb < nbaby) slot = baby0 + bb; }
            T* dst = sm + srow * RS + ev;
            if (slot >= 0 && e0 + ev + V <= total) {
                const T* src = reinterpret_cast<const T*>(base + slot_stride_bytes * slot) + e0 + ev;
                *reinterpret_cast<float4*>(dst) = *reinterpret_cast<const float4*>(src);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) dst[v] = T(0);
            }
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kTPW; ++t) {
            const int tile = warp + t * nwarps;
            if (tile >= ntiles) break;                   // uniform across the warp
            const int g0 = 4 * (tile / nb4), b0 = 4 * ng4 + 4 * (tile % nb4);
            T c16[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) c16[q] = T(0);
            for (int e = lane; e < kChunk; e += 32) {
                T gv[4], bv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) gv[a] = sm[(g0 + a) * RS + e];
#pragma unroll
                for (int b = 0; b < 4; ++b) bv[b] = sm[(b0 + b) * RS + e];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) c16[4 * a + b] = fma(gv[a], bv[b], c16[4 * a + b]);
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                if (sizeof(T) == 4) {
                    const T y = c16[q] - cmp[t][q];
                    const T s2 = acc[t][q] + y;
                    cmp[t][q] = (s2 - acc[t][q]) - y;
                    acc[t][q] = s2;
                } else {
                    acc[t][q] += c16[q];
                }
            }
        }
        __syncthreads();
    }
    const int npairs = ngiant * nbaby;
#pragma unroll
    for (int t = 0; t < kTPW; ++t) {
        const int tile = warp + t * nwarps;
        if (tile >= ntiles) break;
        const int tg = tile / nb4, tb = tile % nb4;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            double v = (double)acc[t][q] - (double)cmp[t][q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            const int g = 4 * tg + q / 4, b = 4 * tb + q % 4;
            if (lane == 0 && g < ngiant && b < nbaby)
                partials[(int64_t)blockIdx.x * npairs + g * nbaby + b] = v;
        }
    }
}

__global__ void k_sum_partials(const double* partials, int nblocks, int npairs, double* out) {
    const int pq = blockIdx.x * blockDim.x + threadIdx.x;
    if (pq >= npairs) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(int64_t)b * npairs + pq];
    out[pq] = s;
}

// tau[0..n_terms) from baby traces diag[0..k) (T_1..T_k), giant traces diag[k + l - 2]
// (T_{lk}, l = 2..m-1) and gram[(l-1)*(k-1) + (i-1)] = <T_{lk}, T_i> (l = 1..m-1,
// i = 1..k-1) through tau_{lk+i} = 2 <T_{lk}, T_i> - tau_{lk-i} (Eq. identity).
__global__ void k_assemble_moments(const double* diag, const double* gram, int k, int m,
                                   int n_terms, double n, double* tau) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    tau[0] = n;
    for (int i = 1; i <= k && i < n_terms; ++i) tau[i] = diag[i - 1];
    for (int l = 1; l < m; ++l) {
        const int base = l * k;
        if (base >= n_terms) break;
        if (l >= 2) tau[base] = diag[k + l - 2];
        for (int i = 1; i < k && base + i < n_terms; ++i)
            tau[base + i] = 2.0 * gram[(l - 1) * (k - 1) + (i - 1)] - tau[base - i];
    }
}

// ------------------------------------------------------------ trace and ||P||_F^2
__global__ void k_trace_frob_part(const double* __restrict__ P, int64_t n, int64_t ldp,
                                  double* partials) {
    __shared__ double sh[33];
    double tr = 0.0, fr = 0.0;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const double* row = P + r * ldp;
        for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
            const double v = row[c];
            fr = fma(v, v, fr);
            if (c == r) tr += v;
        }
    }
    tr = block_sum(tr, sh);
    fr = block_sum(fr, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = tr;
        partials[2 * blockIdx.x + 1] = fr;
    }
}

__global__ void k_trace_frob_final(const double* partials, int nparts, DevResult* res) {
    if (threadIdx.x != 0) return;
    double tr = 0.0, fr = 0.0;
    for (int b = 0; b < nparts; ++b) {
        tr += partials[2 * b];
        fr += partials[2 * b + 1];
    }
    res->trace = tr;
    res->frob2 = fr;
}

__global__ void k_copy_out(const double* __restrict__ R, int64_t np, int64_t n,
                           double* __restrict__ P, int64_t ldp) {
    const int64_t total = n * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / n, c = idx - r * n;
        P[r * ldp + c] = R[r * np + c];
    }
}

__global__ void k_copy_out_f32(const float* __restrict__ R, int64_t np, int64_t n,
                               double* __restrict__ P, int64_t ldp) {
    const int64_t total = n * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / n, c = idx - r * n;
        P[r * ldp + c] = (double)R[r * np + c];
    }
}

int grid_for(int64_t total, int threads) {
    int64_t b = (total + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

cudaError_t launch_gershgorin(const double* H, int64_t n, int64_t ld, double* part_lo,
                              double* part_hi, int* part_bad, int nparts, DevResult* res,
                              int use_given, double emin, double emax, cudaStream_t s) {
    if (use_given) {
        k_set_bounds<<<1, 1, 0, s>>>(res, emin, emax);
        return cudaGetLastError();
    }
    k_gershgorin_rows<<<nparts, 256, 0, s>>>(H, n, ld, part_lo, part_hi, part_bad);
    k_gershgorin_final<<<1, 256, 0, s>>>(part_lo, part_hi, part_bad, nparts, res);
    return cudaGetLastError();
}

cudaError_t launch_set_bounds(DevResult* res, double emin, double emax, cudaStream_t s) {
    k_set_bounds<<<1, 1, 0, s>>>(res, emin, emax);
    return cudaGetLastError();
}

cudaError_t launch_set_scalar(double* dst, double v, cudaStream_t s) {
    k_set_scalar<<<1, 1, 0, s>>>(dst, v);
    return cudaGetLastError();
}

cudaError_t launch_export_bounds(const DevResult* res, double* out3, cudaStream_t s) {
    k_export_bounds<<<1, 1, 0, s>>>(res, out3);
    return cudaGetLastError();
}

cudaError_t launch_scale_f64(const double* H, int64_t n, int64_t ld, const DevResult* res,
                             double* X, int64_t np, cudaStream_t s, int* dbg) {
    const int64_t tn = np / 32;
    MatF32 none{nullptr, nullptr, 0, 0};
    k_scale_sym<true><<<(unsigned)(tn * (tn + 1) / 2), 256, 0, s>>>(H, n, ld, res, X, none, np, 0, 0, 1.0f, dbg);
    return cudaGetLastError();
}

cudaError_t launch_scale_split(const double* H, int64_t n, int64_t ld, const DevResult* res,
                               MatF32 X, int64_t np, int planes, int fp16, float pscale,
                               cudaStream_t s, int* dbg) {
    const int64_t tn = np / 32;
    k_scale_sym<false><<<(unsigned)(tn * (tn + 1) / 2), 256, 0, s>>>(H, n, ld, res, nullptr, X, np,
                                                                     planes, fp16, pscale, dbg);
    return cudaGetLastError();
}

cudaError_t launch_pack_f32(const float* A, int64_t n, int64_t lda, MatF32 X, int64_t np,
                            int planes, int fp16, float pscale, cudaStream_t s) {
    k_pack_f32<<<grid_for(np * np, 256), 256, 0, s>>>(A, n, lda, X, np, planes, fp16, pscale);
    return cudaGetLastError();
}

cudaError_t launch_diag_sums(const void* base, int64_t slot_stride_bytes, int count, int64_t n,
                             int64_t np, int is_f64, double* out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    k_diag_sums<<<count, 256, 0, s>>>(reinterpret_cast<const char*>(base), slot_stride_bytes, n,
                                      np, is_f64, out);
    return cudaGetLastError();
}

int gram_blocks(int64_t np, int ngiant, int nbaby) {
    (void)ngiant;
    (void)nbaby;
    const int64_t nchunks = (np * np + kChunk - 1) / kChunk;
    int64_t b = 152 * 4;
    if (b > nchunks) b = nchunks;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_gram(const void* base, int64_t slot_stride_bytes, int giant0, int ngiant,
                        int baby0, int nbaby, int64_t np, int is_f64, double* partials,
                        int max_blocks, double* out, cudaStream_t s) {
    if (ngiant <= 0 || nbaby <= 0) return cudaSuccess;
    if (nbaby > 32) return cudaErrorInvalidValue;
    const int threads = 512;
    const int max_tiles = (threads / 32) * kTPW;
    const int nb4 = (nbaby + 3) / 4;
    const int gmax = 4 * (max_tiles / nb4);           // giants per launch
    if (ngiant > gmax) {
        // giant-major output: one launch per group of giants
        for (int g = 0; g < ngiant; g += gmax) {
            const int ng = ngiant - g < gmax ? ngiant - g : gmax;
            cudaError_t e = launch_gram(base, slot_stride_bytes, giant0 + g, ng, baby0, nbaby, np,
                                        is_f64, partials, max_blocks, out + (int64_t)g * nbaby, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const int ng4 = (ngiant + 3) / 4;
    const size_t elem = is_f64 ? 8 : 4;
    const size_t smem = (size_t)4 * (ng4 + nb4) * (kChunk + kRowPad) * elem;
    int blocks = gram_blocks(np, ngiant, nbaby);
    if (blocks > max_blocks) blocks = max_blocks;
    const char* b = reinterpret_cast<const char*>(base);
    if (is_f64) {
        cudaFuncSetAttribute(k_gram<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_gram<double><<<blocks, threads, smem, s>>>(b, slot_stride_bytes, giant0, ngiant, baby0,
                                                      nbaby, np * np, partials);
    } else {
        cudaFuncSetAttribute(k_gram<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_gram<float><<<blocks, threads, smem, s>>>(b, slot_stride_bytes, giant0, ngiant, baby0,
                                                     nbaby, np * np, partials);
    }
    const int npairs = ngiant * nbaby;
    k_sum_partials<<<(npairs + 127) / 128, 128, 0, s>>>(partials, blocks, npairs, out);
    return cudaGetLastError();
}

cudaError_t launch_assemble_moments(const double* diag, const double* gram, int k, int m,
                                    int n_terms, int64_t n, double* tau, cudaStream_t s) {
    k_assemble_moments<<<1, 32, 0, s>>>(diag, gram, k, m, n_terms, (double)n, tau);
    return cudaGetLastError();
}

cudaError_t launch_trace_frob(const double* P, int64_t n, int64_t ldp, double* partials,
                              int nparts, DevResult* res, cudaStream_t s) {
    k_trace_frob_part<<<nparts, 256, 0, s>>>(P, n, ldp, partials);
    k_trace_frob_final<<<1, 32, 0, s>>>(partials, nparts, res);
    return cudaGetLastError();
}

cudaError_t launch_copy_out(const double* R, int64_t np, int64_t n, double* P, int64_t ldp,
                            cudaStream_t s) {
    k_copy_out<<<grid_for(n * n, 256), 256, 0, s>>>(R, np, n, P, ldp);
    return cudaGetLastError();
}

cudaError_t launch_copy_out_f32(const float* R, int64_t np, int64_t n, double* P, int64_t ldp,
                                cudaStream_t s) {
    k_copy_out_f32<<<grid_for(n * n, 256), 256, 0, s>>>(R, np, n, P, ldp);
    return cudaGetLastError();
}

}  // namespace fo
