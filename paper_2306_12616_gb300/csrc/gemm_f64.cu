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

// Grouped over the batch and over the steps of a stage: block b covers symmetric tile
// (b mod tiles) - pre[i] of instance i for step b / tiles.
__global__ void __launch_bounds__(256) k_gemm_f64(const __grid_constant__ StepList steps,
                                                  const Inst* __restrict__ insts,
                                                  const InstIO* __restrict__ io, Work wt) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN];
    const int sidx = blockIdx.x / wt.total;
    const int bt = blockIdx.x - sidx * wt.total;
    const Step& st = steps.s[sidx];
    const int inst = find_inst(wt.pre, 0, wt.count, bt);
    const Inst& in = insts[inst];
    if (!step_needed(in.res, st.need_m)) return;
    const int64_t np = in.np;
    const int n_real = (int)in.n;
    const int64_t sb = in.slot_bytes;
    const double* A = reinterpret_cast<const double*>(in.slots + sb * st.a);
    const double* B = reinterpret_cast<const double*>(in.slots + sb * st.b);
    const double* C = st.c >= 0 ? reinterpret_cast<const double*>(in.slots + sb * st.c) : nullptr;
    const double* D = st.d >= 0 ? reinterpret_cast<const double*>(in.slots + sb * st.d) : nullptr;
    double* out = st.out >= 0 ? reinterpret_cast<double*>(in.slots + sb * st.out) : nullptr;
    double* out64 = st.out64 ? io[inst].P : nullptr;
    const int64_t ldo = io[inst].ldp;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int t = (int)(np / BM);
    int I, J;
    upper_tile(bt - wt.pre[inst], t, I, J);
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
            double a[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
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
            double v = st.alpha64 * acc[i][j];
            if (C) v = fma(st.beta64, C[o], v);
            if (D) v += D[o];
            if (r == c && r < n_real) v += st.shift64;
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

int64_t f64_tiles(int64_t np) {
    const int64_t t = np / BM;
    return t * (t + 1) / 2;
}

cudaError_t launch_gemm_f64(const Step* steps, int nsteps, const Inst* in, const InstIO* io, Work wt,
                            cudaStream_t s) {
    if (nsteps < 1 || nsteps > kMaxSteps) return cudaErrorInvalidValue;
    StepList sl;
    for (int q = 0; q < nsteps; ++q) sl.s[q] = steps[q];
    sl.count = nsteps;
    k_gemm_f64<<<(unsigned)wt.total * nsteps, 256, 0, s>>>(sl, in, io, wt);
    return cudaGetLastError();
}

}  // namespace fo
