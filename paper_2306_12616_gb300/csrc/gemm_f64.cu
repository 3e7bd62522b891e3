// Float64 recurrence product out = alpha * A B + beta * C + D + shift * I_n (plain path).
//
// tcgen05 has no float64 kind, so the float64 path runs on the DFMA pipe: 64 x 64 output
// tiles, 16-deep k slices staged in shared memory, 4 x 4 outputs per thread. The update of
// the three-term recurrence (2 T_1 T_i - T_{i-1}) and of the Clenshaw giant steps
// (2 Y b_{l+1} - b_{l+2} + R_l) is applied in the epilogue, so every step is one launch.
// Products of polynomials in the symmetric X are symmetric: only tiles on or above the
// diagonal are launched and each result is stored at (r, c) and (c, r), which halves the
// DFMA work and keeps every stored matrix exactly symmetric.
#include "internal.cuh"

namespace fo {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

__global__ void __launch_bounds__(256) k_gemm_f64(const double* __restrict__ A,
                                                  const double* __restrict__ B, int64_t np,
                                                  double alpha, const double* __restrict__ C,
                                                  double beta, const double* __restrict__ D,
                                                  double shift, int n_real,
                                                  double* __restrict__ out,
                                                  double* __restrict__ out64, int64_t ldo) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int t = (int)(np / BM);
    int I = 0, b = blockIdx.x;
    while (b >= t - I) { b -= t - I; ++I; }
    const int J = I + b;
    const int64_t m0 = (int64_t)I * BM, n0 = (int64_t)J * BN;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    for (int64_t k0 = 0; k0 < np; k0 += BK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = threadIdx.x + 256 * q;
            const int ar = idx >> 4, ac = idx & 15;
            As[ac][ar] = A[(m0 + ar) * np + k0 + ac];
            const int br = idx >> 6, bc = idx & 63;
            Bs[br][bc] = B[(k0 + br) * np + n0 + bc];
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = m0 + ty + 16 * i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t c = n0 + tx + 16 * j;
            const int64_t o = r * np + c;
            double v = alpha * acc[i][j];
            if (C) v = fma(beta, C[o], v);
            if (D) v += D[o];
            if (r == c && r < n_real) v += shift;
            if (c < r) continue;            // lower triangle: written by the mirror
            if (out64) {
                if (r < n_real && c < n_real) {
                    out64[r * ldo + c] = v;
                    if (c > r) out64[c * ldo + r] = v;
                }
            } else {
                out[o] = v;
                if (c > r) out[c * np + r] = v;
            }
        }
    }
}

}  // namespace

cudaError_t launch_gemm_f64(const double* A, const double* B, int64_t np, double alpha,
                            const double* C, double beta, const double* D, double shift,
                            int n_real, double* out, double* out64, int64_t ldo,
                            cudaStream_t s) {
    if (np % BM != 0) return cudaErrorInvalidValue;
    const int64_t t = np / BM;
    k_gemm_f64<<<(unsigned)(t * (t + 1) / 2), 256, 0, s>>>(A, B, np, alpha, C, beta, D, shift, n_real, out, out64, ldo);
    return cudaGetLastError();
}

}  // namespace fo
