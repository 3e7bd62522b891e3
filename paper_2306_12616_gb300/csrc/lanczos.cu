// Lanczos spectral bounds: the tighter alternative to the Gershgorin discs.
//
// The expansion maps H onto [-1, 1] with its lowest and highest eigenvalues (Sec.
// "Chebyshev expansions with O(sqrt L) number of matrix multiplications"); Gershgorin discs
// enclose the spectrum but are several times wider than it for the tight-binding model, which
// costs resolution per term. K steps of the Lanczos process (float64, no reorthogonalisation:
// only the extreme Ritz values are used) give the extreme eigenvalues of the tridiagonal T_K;
// each is widened by its residual beta_{K+1} |y_K| (an eigenvalue of H lies that close) and by
// 1% of the width, and the result is intersected with the Gershgorin interval.
//
// Start vector: v_i = u_i - 1/2, u_i the i-th output of splitmix64 (Steele, Lea and Flood
// 2014) from a fixed seed, scaled to [0, 1): a counter-based draw, identical on any device.
#include "internal.cuh"

namespace fo {
namespace {

constexpr uint64_t kLzSeed = 0x4C414E43ull;
constexpr double kLzMargin = 0.01;

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum_d(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < nw ? sh[lane] : 0.0;
        t = warp_sum_d(t);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

// i-th splitmix64 output of the stream started at seed, in [0, 1).
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// Per-instance state at in.lz: q_prev[np], q[np], w[np], alpha[kLzMax], beta[kLzMax + 1],
// steps done, stopped flag.
struct Lz {
    double *qp, *q, *w, *alpha, *beta, *meta;
};
__device__ __forceinline__ Lz lz_of(const Inst& in) {
    Lz z;
    z.qp = in.lz;
    z.q = z.qp + in.np;
    z.w = z.q + in.np;
    z.alpha = z.w + in.np;
    z.beta = z.alpha + kLzMax;
    z.meta = z.beta + kLzMax + 1;
    return z;
}

__global__ void k_lz_init(const Inst* __restrict__ insts, int batch) {
    __shared__ double sh[33];
    const Inst& in = insts[blockIdx.x];
    const Lz z = lz_of(in);
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < in.np; i += blockDim.x) {
        const double v = i < in.n ? splitmix_uniform(kLzSeed, (uint64_t)i) - 0.5 : 0.0;
        z.q[i] = v;
        z.qp[i] = 0.0;
        s = fma(v, v, s);
    }
    s = block_sum_d(s, sh);
    const double inv = 1.0 / sqrt(s);
    for (int64_t i = threadIdx.x; i < in.np; i += blockDim.x) z.q[i] *= inv;
    if (threadIdx.x == 0) {
        z.beta[0] = 0.0;
        z.meta[0] = 0.0;   // steps done
        z.meta[1] = 0.0;   // stopped
    }
}

// w = H q - beta_j q_prev for the rows of this block (a warp per row); partial w . q.
__global__ void __launch_bounds__(32 * kGershRows) k_lz_matvec(const Inst* __restrict__ insts,
                                                               const InstIO* __restrict__ io, Work wg, int j,
                                                               double* part) {
    __shared__ double sp[kGershRows];
    const int b = blockIdx.x;
    const int i = find_inst(wg.pre, 0, wg.count, b);
    const Inst& in = insts[i];
    const Lz z = lz_of(in);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = in.n, ld = io[i].ldh;
    const int64_t row = (int64_t)(b - wg.pre[i]) * kGershRows + warp;
    double d = 0.0;
    if (z.meta[1] == 0.0 && row < n) {
        const double* hr = io[i].H + row * ld;
        double s = 0.0;
        for (int64_t c = lane; c < n; c += 32) s = fma(__ldg(hr + c), z.q[c], s);
        s = warp_sum_d(s);
        const double wv = s - z.beta[j] * z.qp[row];
        if (lane == 0) z.w[row] = wv;
        d = wv * z.q[row];
    }
    if (lane == 0) sp[warp] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kGershRows; ++w) t += sp[w];
        part[b] = t;
    }
}

// alpha_j, w -= alpha_j q, beta_{j+1} = ||w||, q_prev = q, q = w / beta_{j+1}; one block per
// instance. Stops (for good) on an invariant subspace.
__global__ void k_lz_update(const Inst* __restrict__ insts, Work wg, int j, const double* part) {
    __shared__ double sh[33];
    const int i = blockIdx.x;
    const Inst& in = insts[i];
    const Lz z = lz_of(in);
    if (z.meta[1] != 0.0) return;
    double a = 0.0;
    if (threadIdx.x == 0)
        for (int b = wg.pre[i]; b < wg.pre[i + 1]; ++b) a += part[b];
    if (threadIdx.x == 0) sh[0] = a;
    __syncthreads();
    a = sh[0];
    __syncthreads();
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < in.n; r += blockDim.x) {
        const double wv = z.w[r] - a * z.q[r];
        z.w[r] = wv;
        s = fma(wv, wv, s);
    }
    const double bnext = sqrt(block_sum_d(s, sh));
    // an invariant subspace, or n steps (the whole space)
    const bool stop = !(bnext > 1e-12 * (fabs(a) + z.beta[j])) || j + 1 >= in.n;
    for (int64_t r = threadIdx.x; r < in.n && !stop; r += blockDim.x) {
        z.qp[r] = z.q[r];
        z.q[r] = z.w[r] / bnext;
    }
    if (threadIdx.x == 0) {
        z.alpha[j] = a;
        z.beta[j + 1] = bnext;
        z.meta[0] = (double)(j + 1);
        if (stop) z.meta[1] = 1.0;
    }
}

// Number of eigenvalues of the K x K tridiagonal (alpha, beta[1..K-1]) below x (Sturm).
__device__ int sturm_count(const double* alpha, const double* beta, int K, double x) {
    int c = 0;
    double d = alpha[0] - x;
    if (d < 0.0) ++c;
    for (int j = 1; j < K; ++j) {
        if (d == 0.0) d = 1e-300;
        d = (alpha[j] - x) - beta[j] * beta[j] / d;
        if (d < 0.0) ++c;
    }
    return c;
}

// |last component| of the unit eigenvector for the eigenvalue theta (forward recurrence,
// the stable direction for an extreme eigenvalue), rescaled against overflow.
__device__ double last_component(const double* alpha, const double* beta, int K, double theta) {
    double ym = 0.0, y = 1.0, nrm = 1.0;
    for (int j = 0; j + 1 < K; ++j) {
        const double yn = ((theta - alpha[j]) * y - (j > 0 ? beta[j] * ym : 0.0)) / beta[j + 1];
        ym = y;
        y = yn;
        nrm += y * y;
        if (nrm > 1e200) {
            const double s = 1e-100;
            y *= s;
            ym *= s;
            nrm *= s * s;
        }
    }
    return fabs(y) / sqrt(nrm);
}

__global__ void k_lz_bounds(const Inst* __restrict__ insts, int batch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    const Inst& in = insts[i];
    const Lz z = lz_of(in);
    DevResult* res = in.res;
    const int K = (int)z.meta[0];
    if (K < 1) return;
    // an enclosure of T's eigenvalues for the bisection
    double lo = INFINITY, hi = -INFINITY;
    for (int j = 0; j < K; ++j) {
        const double r = (j > 0 ? fabs(z.beta[j]) : 0.0) + (j + 1 < K ? fabs(z.beta[j + 1]) : 0.0);
        lo = fmin(lo, z.alpha[j] - r);
        hi = fmax(hi, z.alpha[j] + r);
    }
    double th[2];
    for (int e = 0; e < 2; ++e) {
        const int target = e == 0 ? 1 : K;   // smallest x with count(x) >= target
        double a = lo, b = hi;
        for (int it = 0; it < 200 && b - a > 1e-15 * fmax(1.0, fmax(fabs(a), fabs(b))); ++it) {
            const double mid = 0.5 * (a + b);
            if (sturm_count(z.alpha, z.beta, K, mid) >= target) b = mid;
            else a = mid;
        }
        th[e] = 0.5 * (a + b);
    }
    const double rmin = K > 1 ? z.beta[K] * last_component(z.alpha, z.beta, K, th[0]) : z.beta[K];
    const double rmax = K > 1 ? z.beta[K] * last_component(z.alpha, z.beta, K, th[1]) : z.beta[K];
    const double width = th[1] - th[0];
    double el = th[0] - rmin - kLzMargin * width;
    double eh = th[1] + rmax + kLzMargin * width;
    el = fmax(el, res->bounds[0]);
    eh = fmin(eh, res->bounds[1]);
    if (!(eh - el > 1e-12 * fmax(1.0, fmax(fabs(el), fabs(eh))))) {
        const double c = 0.5 * (el + eh);
        el = c - 1.0;
        eh = c + 1.0;
    }
    if (res->nonfinite) return;   // keep the Gershgorin record of a non-finite H
    res->bounds[0] = el;
    res->bounds[1] = eh;
}

}  // namespace

cudaError_t launch_lanczos(const Inst* in, const InstIO* io, int batch, Work wg, double* part, int steps,
                           cudaStream_t s, int* launches) {
    if (steps < 1) return cudaSuccess;
    if (steps > kLzMax) steps = kLzMax;
    k_lz_init<<<batch, 256, 0, s>>>(in, batch);
    for (int j = 0; j < steps; ++j) {
        k_lz_matvec<<<wg.total, 32 * kGershRows, 0, s>>>(in, io, wg, j, part);
        k_lz_update<<<batch, 256, 0, s>>>(in, wg, j, part);
    }
    k_lz_bounds<<<(batch + 127) / 128, 128, 0, s>>>(in, batch);
    if (launches) *launches += 2 + 2 * steps;
    return cudaGetLastError();
}

}  // namespace fo
