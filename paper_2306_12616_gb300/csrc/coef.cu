// Coefficient pipeline of the expansion, all float64 on the device:
//   cosine table -> DOS weights from the moments -> bisection for mu -> Fermi values at
//   the Chebyshev-Gauss nodes -> coefficients c_n -> giant-step coefficients g_{i,l} ->
//   contraction R_l = sum_i g_{i,l} T_i.
//
// Chebyshev-Gauss nodes: theta_j = pi (2j+1) / (2M), x_j = cos theta_j. Every cosine the
// pipeline needs is cos(n theta_j) = cos(pi r / (2M)) with r = n (2j+1) mod 4M, so one
// table ct[r] = cospi(r / (2M)), r < 4M, serves the nodes, the DCT and the DOS weights.
#include <cuda_bf16.h>
#include <type_traits>
#include <cuda_fp16.h>

#include "internal.cuh"

namespace fo {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fermi-Dirac function f(e) = 1 / (1 + exp((e - mu)/kT)) (Eq. fermifunc) written as
// (1 - tanh((e - mu)/(2 kT)))/2, which never overflows. tanh(x) rounds to +-1 in float64 for
// |x| >= 19.1, so beyond |x| = 20 f is 0 or 1 (the exact values differ by < 5e-18) and the
// float64 tanh, slow on this GPU, is skipped: most Chebyshev nodes lie many kT away from mu.
__device__ __forceinline__ double fermi(double e, double mu, double inv2kT) {
    const double x = (e - mu) * inv2kT;
    if (x >= 20.0) return 0.0;
    if (x <= -20.0) return 1.0;
    return 0.5 - 0.5 * tanh(x);
}

__global__ void k_cos_table(int M, double* ct) {
    const int64_t total = 4LL * M;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total;
         r += (int64_t)gridDim.x * blockDim.x)
        ct[r] = cospi((double)r / (2.0 * (double)M));
}

// w_j = (1/M) (tau_0 + 2 sum_{n=1}^{n_terms-1} tau_n cos(n theta_j)), so that
// sum_n c_n(mu) tau_n = sum_j f(e_j; mu) w_j for the interpolation coefficients c_n.
// Block (node chunk, instance).
__global__ void k_dos_weights(const Inst* __restrict__ insts, int n_terms, int M,
                              const double* __restrict__ ct) {
    const Inst& in = insts[blockIdx.y];
    if (!in.res->active) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const double* tau = in.tau;
    const int64_t q = 2LL * j + 1, fourM = 4LL * M;
    int64_t r = 0;
    double s = 0.0;
    const int nt = eff_terms(in.res, n_terms);
    for (int n = 1; n < nt; ++n) {
        r += q;
        if (r >= fourM) r -= fourM;
        s = fma(tau[n], ct[r], s);
    }
    in.w[j] = (tau[0] + 2.0 * s) / (double)M;
}

// F(mu) + N_e = sum_j w_j f(e_j; mu) and dF/dmu = sum_j w_j f_j (1 - f_j) / kT over the M
// nodes, fixed summation order, both broadcast to the block.
__device__ void trace_at(double mu, const double* __restrict__ w, const double* __restrict__ ct,
                         int M, double mid, double half, double inv2kT, double* sh, double* tr,
                         double* dtr) {
    double s = 0.0, d = 0.0;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const double f = fermi(mid + half * ct[2 * j + 1], mu, inv2kT);
        s = fma(w[j], f, s);
        d = fma(w[j], f * (1.0 - f), d);
    }
    s = warp_sum(s);
    d = warp_sum(d);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) { sh[warp] = s; sh[32 + warp] = d; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, u = 0.0;
        for (int i = 0; i < nw; ++i) { t += sh[i]; u += sh[32 + i]; }
        sh[64] = t;
        sh[65] = u * 2.0 * inv2kT;
    }
    __syncthreads();
    *tr = sh[64];
    if (dtr) *dtr = sh[65];
}

// Root of F(mu) = sum_n c_n(mu) tau_n - N_e, one block per instance. Bracket [emin, emax],
// widened by 10 kT (at most 8 times per side). Inside the bracket a Newton step on the
// exact derivative of the node sum is taken when it stays in the bracket and is at most
// half the step before the last one, a halving otherwise; the bracket shrinks with the sign
// of F at every evaluated point. The first
// point is the midpoint, or res->mu0 when start_mu0 is set and mu0 lies inside the
// bracket (the learned proposal). Stop when |F| <= 1e-12 max(1, N_e) (mu = that point) or
// the bracket is narrower than 1e-15 (emax - emin) (mu = midpoint), at most max_iter
// evaluations.
__global__ void __launch_bounds__(512) k_bisect(const Inst* __restrict__ insts,
                                                 const InstIO* __restrict__ io,
                                                 const double* __restrict__ ct, int M,
                                                 int max_iter, int start_mu0) {
    __shared__ double sh[66];
    const Inst& in = insts[blockIdx.x];
    DevResult* res = in.res;
    if (!res->active) return;
    const double* w = in.w;
    const double kT = io[blockIdx.x].kT, n_e = io[blockIdx.x].n_e;
    const double ea = res->bounds[0], eb = res->bounds[1];
    const double mid = 0.5 * (eb + ea), half = 0.5 * (eb - ea), inv2kT = 0.5 / kT;
    double lo = ea, hi = eb, t;
    // F at the bracket ends, from the widening loops (evaluated again only where a loop ended
    // by widening past its last evaluation)
    double flo = 1.0, fhi = -1.0;
    bool have_lo = false, have_hi = false;
    for (int q = 0; q < 8; ++q) {
        trace_at(lo, w, ct, M, mid, half, inv2kT, sh, &t, nullptr);
        if (t - n_e <= 0.0) { flo = t - n_e; have_lo = true; break; }
        lo -= 10.0 * kT;
    }
    for (int q = 0; q < 8; ++q) {
        trace_at(hi, w, ct, M, mid, half, inv2kT, sh, &t, nullptr);
        if (t - n_e >= 0.0) { fhi = t - n_e; have_hi = true; break; }
        hi += 10.0 * kT;
    }
    if (!have_lo) { trace_at(lo, w, ct, M, mid, half, inv2kT, sh, &flo, nullptr); flo -= n_e; }
    if (!have_hi) { trace_at(hi, w, ct, M, mid, half, inv2kT, sh, &fhi, nullptr); fhi -= n_e; }
    int status = FO_OK, iters = 0;
    double mu = 0.5 * (lo + hi);
    if (flo > 0.0 || fhi < 0.0) {
        status = FO_ERR_NO_BRACKET;
    } else {
        const double tol_f = 1e-12 * fmax(1.0, fabs(n_e));
        const double tol_w = 1e-15 * (eb - ea);
        bool done = false;
        double x = 0.5 * (lo + hi);
        if (start_mu0 && res->mu0 > lo && res->mu0 < hi) x = res->mu0;
        // the last two steps: a Newton step is taken only when it is at most half the step
        // before the last one (near the root the rounding of F can make Newton steps stall on
        // one side, each moving one end of the bracket by a tiny amount; quadratic convergence
        // passes this test)
        double dx = hi - lo, dxold = dx;
        for (int it = 1; it <= max_iter; ++it) {
            double f, df;
            trace_at(x, w, ct, M, mid, half, inv2kT, sh, &f, &df);
            f -= n_e;
            iters = it;
            if (fabs(f) <= tol_f) { mu = x; done = true; break; }
            if (f < 0.0) lo = x; else hi = x;
            if (hi - lo <= tol_w) { mu = 0.5 * (lo + hi); done = true; break; }
            const double cand = (df > 0.0) ? x - f / df : lo;
            const double xn = (cand > lo && cand < hi && fabs(cand - x) <= 0.5 * fabs(dxold)) ? cand : 0.5 * (lo + hi);
            dxold = dx;
            dx = xn - x;
            x = xn;
        }
        if (!done) {
            mu = 0.5 * (lo + hi);
            status = FO_ERR_NOT_CONVERGED;
        }
    }
    if (threadIdx.x == 0) {
        res->mu = mu;
        res->iters = iters;
        res->mu_lo = lo;
        res->mu_hi = hi;
        if (res->status == FO_OK) res->status = status;
    }
}

// mu of FO_MU_FIXED from the per-call inputs.
__global__ void k_set_mu(const Inst* __restrict__ insts, const InstIO* __restrict__ io, int batch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < batch) insts[i].res->mu = io[i].mu;
}

// f_j = f(e_j; mu) at the nodes e_j = mid + half x_j, mu read from the device record.
// Block (node chunk, instance).
__global__ void k_fermi_nodes(const Inst* __restrict__ insts, const InstIO* __restrict__ io, int M,
                              const double* __restrict__ ct) {
    const Inst& in = insts[blockIdx.y];
    const DevResult* res = in.res;
    if (!res->active) return;
    // 1 / (2 kT) once per block (a float64 division per node would dominate this kernel)
    __shared__ double s_inv2kT;
    if (threadIdx.x == 0) s_inv2kT = 0.5 / io[blockIdx.y].kT;
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const double ea = res->bounds[0], eb = res->bounds[1];
    in.f[j] = fermi(0.5 * (eb + ea) + 0.5 * (eb - ea) * ct[2 * j + 1], res->mu, s_inv2kT);
}

// c_n = (2 - delta_{n0}) / M sum_j f_j cos(n theta_j) for n < n_terms, 0 for n_terms <= n < km.
// One warp per n; block (warp group, instance).
__global__ void k_coeffs(const Inst* __restrict__ insts, const double* __restrict__ ct, int M,
                         int n_terms, int km) {
    const Inst& in = insts[blockIdx.y];
    if (!in.res->active) return;
    const int lane = threadIdx.x & 31;
    const int n = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (n >= km) return;
    double* c = in.c;
    if (n >= eff_terms(in.res, n_terms)) {
        if (lane == 0) c[n] = 0.0;
        return;
    }
    const double* f = in.f;
    const int64_t fourM = 4LL * M;
    double s = 0.0;
    for (int j = lane; j < M; j += 32) {
        const int64_t r = ((int64_t)n * (2LL * j + 1)) % fourM;
        s = fma(f[j], ct[r], s);
    }
    s = warp_sum(s);
    if (lane == 0) c[n] = (n == 0 ? 1.0 : 2.0) * s / (double)M;
}

// Giant-step coefficients from c (zero-padded to km), g stored l-major: g[l*k + i].
// c_{lk} = g_{0,l}; c_i = g_{i,0} + g_{k-i,1}/2; c_{lk+i} = (g_{i,l} + g_{k-i,l+1})/2 for
// 1 <= l <= m-2; c_{(m-1)k+i} = g_{i,m-1}/2; c_i = g_{i,0} if m = 1. Solved downwards in l.
// One block per instance.
__global__ void k_g_convert(const Inst* __restrict__ insts, int k, int m) {
    const Inst& in = insts[blockIdx.x];
    if (!in.res->active) return;
    const double* c = in.c;
    double* g = in.g;
    for (int l = m - 1; l >= 0; --l) {
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            const double ci = c[l * k + i];
            double v;
            if (i == 0 || m == 1) v = ci;
            else if (l == m - 1) v = 2.0 * ci;
            else if (l == 0) v = ci - 0.5 * g[1 * k + (k - i)];
            else v = 2.0 * ci - g[(l + 1) * k + (k - i)];
            g[l * k + i] = v;
        }
        __syncthreads();
    }
}

// The paper's power-basis coefficients d_{i,j} of P = sum_j T_k^j S_j, S_j = sum_i d_{i,j} T_i
// (Eq. ansatz), from the giant-step coefficients: T_{lk} = T_l(T_k) = sum_j t_{l,j} T_k^j with
// t_{l,j} the monomial coefficients of the Chebyshev polynomial T_l (t_{l+1,j} = 2 t_{l,j-1} -
// t_{l-1,j}), so d_{i,j} = sum_l g_{i,l} t_{l,j}, i.e. D = G A^{-1} for the A of Eq. (coeff
// recursion). Written over g in place; one block per instance, the table in shared memory.
__global__ void k_g_to_d(const Inst* __restrict__ insts, int k, int m) {
    extern __shared__ double sm_t[];   // t[l * m + j], m x m, then g[k x m]
    const Inst& in = insts[blockIdx.x];
    if (!in.res->active) return;
    double* t = sm_t;
    double* gs = sm_t + m * m;
    for (int q = threadIdx.x; q < m * m; q += blockDim.x) t[q] = 0.0;
    for (int q = threadIdx.x; q < k * m; q += blockDim.x) gs[q] = in.g[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        t[0] = 1.0;
        if (m > 1) t[m + 1] = 1.0;
        for (int l = 1; l + 1 < m; ++l)
            for (int j = 0; j <= l + 1; ++j)
                t[(l + 1) * m + j] = (j > 0 ? 2.0 * t[l * m + j - 1] : 0.0) - t[(l - 1) * m + j];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < k * m; q += blockDim.x) {
        const int j = q / k, i = q - j * k;   // g and d stored l-major: [l * k + i]
        double s = 0.0;
        for (int l = j; l < m; ++l) s = fma(gs[l * k + i], t[l * m + j], s);
        in.g[j * k + i] = s;
    }
}

__global__ void k_poly_trace(const Inst* __restrict__ insts, int n_terms) {
    const Inst& in = insts[blockIdx.x];
    if (!in.res->active) return;
    double s = 0.0;
    const int nt = eff_terms(in.res, n_terms);
    for (int n = threadIdx.x; n < nt; n += 32) s = fma(in.c[n], in.tau[n], s);
    s = warp_sum(s);
    if (threadIdx.x == 0) in.res->trace_poly = s;
}

// Effective temperature of the truncated expansion p(e) = sum_n c_n T_n(x(e)) at the current
// mu: kT_p = integral of p (1 - p) de over [e_a, e_b]. For the Fermi function itself the
// integral is exactly kT; a truncated expansion smears the step over a wider range (about
// the width divided by the number of terms), and d tr P / d mu ~ tr(P - P^2) / kT_p then
// holds where tr(P - P^2) / kT overstates the slope. Gauss-Chebyshev rule on the nodes:
// de = (e_b - e_a)/2 sin(theta) dtheta, p_j = sum_n c_n cos(n theta_j). One block per
// instance.
__global__ void __launch_bounds__(256) k_poly_width(const Inst* __restrict__ insts, const double* __restrict__ ct,
                                                    int M, int n_terms) {
    const Inst& in = insts[blockIdx.x];
    DevResult* res = in.res;
    if (!res->active) return;
    const int64_t fourM = 4LL * M;
    const double* c = in.c;
    double acc = 0.0;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const int64_t step = 2LL * j + 1;
        int64_t r = 0;
        double p = 0.0;
        for (int n = 0; n < n_terms; ++n) {
            p = fma(c[n], ct[r], p);
            r += step;
            if (r >= fourM) r -= fourM;
        }
        const int64_t rs = (step - M + fourM) % fourM;    // sin(theta_j) = cos(theta_j - pi/2)
        acc = fma(ct[rs], p * (1.0 - p), acc);
    }
    __shared__ double part[8];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        res->kt_eff = 0.5 * (res->bounds[1] - res->bounds[0]) * (3.14159265358979323846 / (double)M) * t;
    }
}

// R_l = g_{0,l} I_n + sum_{i=1}^{k-1} g_{i,l} T_i for all l < m, float64. T_i is slot i-1,
// R_l slot n_tslots + l. A block covers ew_rows(np) rows of one instance; outputs are
// produced in groups of kGroup l's per pass over the T_i.
constexpr int kGroup = 16;

__global__ void __launch_bounds__(256) k_contract_f64(const Inst* __restrict__ insts, Work we, int k,
                                                      int m, int n_tslots) {
    extern __shared__ double gsh[];
    const int i = find_inst(we.pre, 0, we.count, blockIdx.x);
    const Inst& in = insts[i];
    if (!in.res->active) return;
    for (int q = threadIdx.x; q < k * m; q += blockDim.x) gsh[q] = in.g[q];
    __syncthreads();
    const int64_t np = in.np, n = in.n;
    const int rows = ew_rows(np);
    const int64_t r0 = (int64_t)(blockIdx.x - we.pre[i]) * rows;
    const int64_t r1 = r0 + rows < np ? r0 + rows : np;
    const int64_t tstride = in.slot_bytes / 8;
    const double* tbase = reinterpret_cast<const double*>(in.slots);
    double* rbase = reinterpret_cast<double*>(in.slots + n_tslots * in.slot_bytes);
    for (int64_t idx = r0 * np + threadIdx.x; idx < r1 * np; idx += blockDim.x) {
        const int64_t r = idx / np, col = idx - r * np;
        const bool diag = (r == col) && (r < n);
        for (int l0 = 0; l0 < m; l0 += kGroup) {
            double acc[kGroup];
#pragma unroll
            for (int q = 0; q < kGroup; ++q) acc[q] = 0.0;
            for (int t = 1; t < k; ++t) {
                const double v = tbase[(int64_t)(t - 1) * tstride + idx];
#pragma unroll
                for (int q = 0; q < kGroup; ++q)
                    if (l0 + q < m) acc[q] = fma(gsh[(l0 + q) * k + t], v, acc[q]);
            }
#pragma unroll
            for (int q = 0; q < kGroup; ++q) {
                if (l0 + q < m) {
                    double v = acc[q];
                    if (diag) v += gsh[(l0 + q) * k];
                    rbase[(int64_t)(l0 + q) * tstride + idx] = v;
                }
            }
        }
    }
}

// float32 version: slots hold a float32 master at element offset 0 and 16-bit planes at
// float offset np*np with plane stride np*np; planes are written for R_{m-1} only (it is
// the first Clenshaw operand). Two entries per thread and step.
__device__ __forceinline__ uint16_t bf16_bits_c(float v) {
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<uint16_t*>(&h);
}

struct Split3 {
    uint16_t p[3];
};
__device__ __forceinline__ Split3 split_value(float v, int fp16, float pscale) {
    Split3 o;
    if (!fp16) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v);
        const float r1 = v - __bfloat162float(h0);
        const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
        o.p[0] = *reinterpret_cast<const uint16_t*>(&h0);
        o.p[1] = *reinterpret_cast<const uint16_t*>(&h1);
        o.p[2] = bf16_bits_c(r1 - __bfloat162float(h1));
    } else {
        const float x = v * pscale;
        const __half h0 = __float2half_rn(x);
        const __half h1 = __float2half_rn(x - __half2float(h0));
        o.p[0] = *reinterpret_cast<const uint16_t*>(&h0);
        o.p[1] = *reinterpret_cast<const uint16_t*>(&h1);
        o.p[2] = 0;
    }
    return o;
}

// R_l for l0 <= l < min(l0 + MAXM, m) (MAXM = m rounded up to a multiple of 4, at most 32;
// m > 32 takes several launches), on and above the diagonal only (the float32 masters of the
// T_i are maintained there; R_l is symmetric). The upper triangle is walked as 16-byte quads
// (row r from column 4 floor(r / 4) to the end; ct_quads), one quad per pair of adjacent
// threads and step, consecutive pairs on consecutive quads; quad q of the flattened order lies
// in the row group b = floor(r / 4) with C(b) <= q < C(b + 1), C(b) = b np - 2 b (b - 1),
// found by a square root and corrected exactly. The two threads of a pair stage alternate
// quads of T_1..T_{k-1} into the pair's slots of a two-stage shared-memory ring by cp.async
// (a warp barrier, not a block barrier, publishes them to the partner) and each forms half
// of the R_l from all k - 1 quads with the coefficients, staged as duplicated pairs
// gsh[t][l] = (g_{t,l0+l}, g_{t,l0+l}) (zero beyond m): one 16-byte broadcast load serves two
// R_l, each packed FMA two entries of the quad, and each R_l leaves as one 16-byte store.
// Two threads per quad halve the accumulators per thread and double the warps per SM that
// keep copies in flight. The planes of the instance's last R (R_{m-1}, or R_{m_eff-1} when a
// learned order cut its expansion: the first operand of the Clenshaw steps) are written here
// and completed below the diagonal by k_mirror_planes.
template <int MAXM>
__global__ void __launch_bounds__(128, 4) k_contract_f32(const Inst* __restrict__ insts, Work wct, int k, int m,
                                                          int l0, int n_tslots, int planes_last, int fp16,
                                                          float pscale, int* dbg) {
    static_assert(MAXM % 4 == 0, "l pairs per half");
    constexpr int HM = MAXM / 2;                           // R_l per thread
    extern __shared__ __align__(16) float fsh[];
    const int i = find_inst(wct.pre, 0, wct.count, blockIdx.x);
    const Inst& in = insts[i];
    if (!in.res->active) return;
    const int tid = threadIdx.x;
    const int npr = blockDim.x >> 1;                       // thread pairs: one quad per pair
    const int pr = tid >> 1, h = tid & 1;                  // pair, and which half of the R_l
    for (int q = tid; q < k * MAXM; q += blockDim.x) {
        const int t = q / MAXM, l = l0 + q - t * MAXM;
        const float g = l < m ? (float)in.g[l * k + t] : 0.0f;
        fsh[2 * q] = g;
        fsh[2 * q + 1] = g;
    }
    const int nt = k - 1;                                   // T_1 .. T_{k-1}
    float4* ring = reinterpret_cast<float4*>(fsh + 2 * k * MAXM);   // [stage][t][pair]
    const int64_t np = in.np, n = in.n;
    const int lastl = (in.res->m_eff > 0 ? in.res->m_eff : m) - 1;   // R whose planes are written
    const int64_t q_all = ct_quads(np);
    const int64_t per = (int64_t)npr * kCtSteps;
    const int64_t q0 = (int64_t)(blockIdx.x - wct.pre[i]) * per;
    const int64_t q1 = q0 + per < q_all ? q0 + per : q_all;
    const int nsteps = (int)((q1 - q0 + npr - 1) / npr);
    const int64_t tstride = in.slot_bytes / 4;
    const int64_t ps = np * np;
    const float* tbase = reinterpret_cast<const float*>(in.slots);
    float* rbase = reinterpret_cast<float*>(in.slots + n_tslots * in.slot_bytes);
    // (row, column) of this pair's quad of step j, or row -1 past the block's range. 32-bit
    // integers (n_pad <= 65536: q < n_pad (n_pad + 4) / 8 < 2^31, b n_pad < 2^30), so the
    // division is a short 32-bit one
    const int npi = (int)np, G = npi / 4;                   // row groups
    auto locate = [&](int j, int& r, int& c) {
        const int64_t q64 = q0 + (int64_t)j * npr + pr;
        r = -1;
        c = 0;
        if (q64 >= q1) return;
        const int q = (int)q64;
        const float e = (float)(npi + 2);
        const float d = e * e - 8.0f * (float)q;
        int b = (int)((e - sqrtf(d > 0.0f ? d : 0.0f)) * 0.25f);
        if (b < 0) b = 0;
        if (b > G - 1) b = G - 1;
        auto C = [&](int x) { return x * npi - 2 * x * (x - 1); };
        while (b > 0 && C(b) > q) --b;
        while (b + 1 < G && C(b + 1) <= q) ++b;
        const int len = G - b;                              // quads per row of the group
        const int off = q - C(b);
        const int dr = off / len;
        r = 4 * b + dr;
        c = 4 * b + 4 * (off - dr * len);
    };
    // the pair's quads of T_1..T_{k-1} at (r, c) into stage st: each thread copies every other one
    auto issue = [&](int st, int r, int c) {
        if (r >= 0 && nt > h) {
            float4* dst = ring + (int64_t)st * nt * npr + (int64_t)h * npr + pr;
            const float* src = tbase + (int64_t)r * np + c + (int64_t)h * tstride;   // slot t holds T_{t+1}
#pragma unroll 1
            for (int t = h; t < nt; t += 2, dst += 2 * npr, src += 2 * tstride) cp_async16(dst, src);
        }
        cp_async_commit();
    };
    int r, c;   // the quad of the current step, located when its copies were issued
    locate(0, r, c);
    issue(0, r, c);
    __syncthreads();   // the coefficient table
    const float4* gtab = reinterpret_cast<const float4*>(fsh) + h * (HM / 2);   // [t][l / 2], this half
    for (int j = 0; j < nsteps; ++j) {
        int rn, cn;
        locate(j + 1, rn, cn);
        issue((j + 1) & 1, rn, cn);
        cp_async_wait<1>();   // this thread's copies of step j have landed
        __syncwarp();         // and its partner's: both halves of the pair's quads are visible
        const int64_t idx = (int64_t)r * np + c;
        if (r >= 0 && FO_CHK(dbg, idx >= 0 && idx + 3 < ps && (idx & 3) == 0, 302, r, idx)) {
            const float4* vp = ring + (int64_t)(j & 1) * nt * npr + pr;   // T_1's quad of this pair
            const float4* gp = gtab + MAXM / 2;                             // row t = 1
            float2 acc[HM][2];   // R_{l0 + h HM + l} at entries (0, 1) and (2, 3) of the quad
#pragma unroll
            for (int l = 0; l < HM; ++l) acc[l][0] = acc[l][1] = make_float2(0.0f, 0.0f);
#pragma unroll 2
            for (int t = 0; t < nt; ++t, vp += npr, gp += MAXM / 2) {
                const float4 v = *vp;
                const float2 v01 = make_float2(v.x, v.y), v23 = make_float2(v.z, v.w);
#pragma unroll
                for (int l2 = 0; l2 < HM / 2; ++l2) {
                    const float4 g = gp[l2];   // (g_l, g_l, g_{l+1}, g_{l+1})
                    const float2 ga = make_float2(g.x, g.y), gb = make_float2(g.z, g.w);
                    acc[2 * l2][0] = __ffma2_rn(v01, ga, acc[2 * l2][0]);
                    acc[2 * l2][1] = __ffma2_rn(v23, ga, acc[2 * l2][1]);
                    acc[2 * l2 + 1][0] = __ffma2_rn(v01, gb, acc[2 * l2 + 1][0]);
                    acc[2 * l2 + 1][1] = __ffma2_rn(v23, gb, acc[2 * l2 + 1][1]);
                }
            }
            const int dg = (r < n && c == (r & ~int64_t(3))) ? (int)(r & 3) : -1;   // diagonal entry
            float* dst = rbase + (int64_t)(l0 + h * HM) * tstride + idx;
#pragma unroll
            for (int l = 0; l < HM; ++l, dst += tstride) {
                const int L = l0 + h * HM + l;
                if (L >= m) break;
                float4 v = make_float4(acc[l][0].x, acc[l][0].y, acc[l][1].x, acc[l][1].y);
                if (dg >= 0) {   // g_{0,l}: the t = 0 row (T_0 = I)
                    const float g0 = fsh[2 * (h * HM + l)];
                    if (dg == 0) v.x += g0;
                    else if (dg == 1) v.y += g0;
                    else if (dg == 2) v.z += g0;
                    else v.w += g0;
                }
                *reinterpret_cast<float4*>(dst) = v;
                if (L == lastl && planes_last > 0) {
                    const Split3 s0 = split_value(v.x, fp16, pscale), s1 = split_value(v.y, fp16, pscale);
                    const Split3 s2 = split_value(v.z, fp16, pscale), s3 = split_value(v.w, fp16, pscale);
                    // planes of R_l: 16-bit entries from float offset ps of the slot
                    uint16_t* pl = reinterpret_cast<uint16_t*>(dst - idx + ps) + idx;
#pragma unroll
                    for (int p = 0; p < 3; ++p) {
                        if (p >= planes_last) break;
                        const uint2 w = make_uint2((uint32_t)s0.p[p] | ((uint32_t)s1.p[p] << 16),
                                                   (uint32_t)s2.p[p] | ((uint32_t)s3.p[p] << 16));
                        *reinterpret_cast<uint2*>(pl + p * ps) = w;
                    }
                }
            }
        }
        __syncwarp();   // both threads are done with the pair's ring slot before it is refilled
        r = rn;
        c = cn;
    }
    cp_async_wait<0>();
}

// The 16-bit planes of one slot below the diagonal from those above it: block (bi, bj),
// bj >= bi, of 32 x 32 entries (the enumeration of k_scale_sym) is staged in shared memory
// and written transposed at (bj, bi); a diagonal block fills its own lower half. With ublk
// only the diagonal 128-blocks are completed (a lower 128-block is then read as the
// transpose of its upper counterpart).
__global__ void __launch_bounds__(256) k_mirror_planes(const Inst* __restrict__ insts, Work ws, int slot0, int m,
                                                       int planes, int ublk, int* dbg) {
    __shared__ uint16_t tile[3][32][33];
    const int i = find_inst(ws.pre, 0, ws.count, blockIdx.x);
    if (!insts[i].res->active) return;
    // the instance's last R: R_{m-1}, or R_{m_eff-1} for an expansion cut by a learned order
    const int slot = slot0 + (insts[i].res->m_eff > 0 ? insts[i].res->m_eff : m) - 1;
    const int64_t np = insts[i].np;
    const int tn = (int)(np / 32);
    int bi, bj;
    upper_tile(blockIdx.x - ws.pre[i], tn, bi, bj);
    if (ublk && bi * 32 / kPad != bj * 32 / kPad) return;
    const int64_t ps = np * np;
    // 32-bit words of 16-bit entries (row offsets and tile columns are even)
    uint32_t* P32 = reinterpret_cast<uint32_t*>(insts[i].slots + insts[i].slot_bytes * slot + 4 * ps);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // word of a tile row, row
    for (int pl = 0; pl < planes; ++pl)
        for (int ry = ty; ry < 32; ry += 16) {
            const uint32_t w = P32[(pl * ps + ((int64_t)bi * 32 + ry) * np + (int64_t)bj * 32) / 2 + tx];
            tile[pl][ry][2 * tx] = (uint16_t)(w & 0xffffu);
            tile[pl][ry][2 * tx + 1] = (uint16_t)(w >> 16);
        }
    __syncthreads();
    for (int pl = 0; pl < planes; ++pl)
        for (int ry = ty; ry < 32; ry += 16) {
            // output (bj*32 + ry, bi*32 + 2 tx + e) = input (bi*32 + 2 tx + e, bj*32 + ry), e = 0, 1.
            // Written where the first entry is below the diagonal; the second is then below it
            // or on it, and the diagonal entry is its own transpose (the same value rewritten)
            const int64_t r = (int64_t)bj * 32 + ry, c = (int64_t)bi * 32 + 2 * tx;
            if (r <= c) continue;
            if (!FO_CHK(dbg, r < np && c + 1 < np, 303, r, c)) continue;
            const uint32_t w = (uint32_t)tile[pl][2 * tx][ry] | ((uint32_t)tile[pl][2 * tx + 1][ry] << 16);
            P32[(pl * ps + r * np + c) / 2] = w;
        }
}

int grid_for(int64_t total, int threads) {
    int64_t b = (total + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

cudaError_t launch_cos_table(int M, double* ct, cudaStream_t s) {
    k_cos_table<<<grid_for(4LL * M, 256), 256, 0, s>>>(M, ct);
    return cudaGetLastError();
}

cudaError_t launch_dos_weights(const Inst* in, int batch, const Shape& sh, const double* ct, cudaStream_t s) {
    k_dos_weights<<<dim3((sh.M + 127) / 128, batch), 128, 0, s>>>(in, sh.n_terms, sh.M, ct);
    return cudaGetLastError();
}

cudaError_t launch_bisect(const Inst* in, const InstIO* io, int batch, const Shape& sh, const double* ct,
                          int max_iter, int start_mu0, cudaStream_t s) {
    // four warps per instance: the node sums are few float64 operations per thread, the
    // float64 shuffle trees and the block reduction are per warp (this GPU's float64 pipe is
    // narrow), so fewer warps finish an evaluation sooner
    k_bisect<<<batch, 128, 0, s>>>(in, io, ct, sh.M, max_iter, start_mu0);
    return cudaGetLastError();
}

cudaError_t launch_set_mu(const Inst* in, const InstIO* io, int batch, cudaStream_t s) {
    k_set_mu<<<(batch + 127) / 128, 128, 0, s>>>(in, io, batch);
    return cudaGetLastError();
}

cudaError_t launch_coefficients(const Inst* in, const InstIO* io, int batch, const Shape& sh,
                                const double* ct, int with_poly_trace, cudaStream_t s, int* launches) {
    k_fermi_nodes<<<dim3((sh.M + 255) / 256, batch), 256, 0, s>>>(in, io, sh.M, ct);
    const int warps_per_block = 8;
    k_coeffs<<<dim3((sh.km + warps_per_block - 1) / warps_per_block, batch), 32 * warps_per_block, 0, s>>>(
        in, ct, sh.M, sh.n_terms, sh.km);
    k_g_convert<<<batch, sh.k < 1024 ? ((sh.k + 31) / 32) * 32 : 1024, 0, s>>>(in, sh.k, sh.m);
    int l = 3;
    if (with_poly_trace) {
        k_poly_trace<<<batch, 32, 0, s>>>(in, sh.n_terms);
        ++l;
    }
    if (launches) *launches += l;
    return cudaGetLastError();
}

cudaError_t launch_poly_width(const Inst* in, int batch, const Shape& sh, const double* ct, cudaStream_t s) {
    k_poly_width<<<batch, 256, 0, s>>>(in, ct, sh.M, sh.n_terms);
    return cudaGetLastError();
}

cudaError_t launch_g_to_d(const Inst* in, int batch, const Shape& sh, cudaStream_t s) {
    const size_t smem = sizeof(double) * ((size_t)sh.m * sh.m + (size_t)sh.k * sh.m);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_g_to_d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_g_to_d<<<batch, 256, smem, s>>>(in, sh.k, sh.m);
    return cudaGetLastError();
}

cudaError_t launch_contract(const Inst* in, Work we, Work wct, Work wsym, const Shape& sh, cudaStream_t s, int* dbg) {
    if (sh.is64) {
        const size_t smem = (size_t)sh.k * sh.m * sizeof(double);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_contract_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_contract_f64<<<we.total, 256, smem, s>>>(in, we, sh.k, sh.m, sh.n_tslots);
        return cudaGetLastError();
    }
    const int planes_last = sh.m > 1 ? sh.planes : 0;
    // two ring stages of every pair's k - 1 quads
    const int tpb = ct_threads(sh.k);
    const size_t stage_bytes = (size_t)(sh.k - 1) * tpb * 16;
    auto go = [&](auto kern, int maxm, int l0) {
        const size_t smem = (size_t)2 * sh.k * maxm * sizeof(float) + 2 * stage_bytes;
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<wct.total, 2 * tpb, smem, s>>>(in, wct, sh.k, sh.m, l0, sh.n_tslots, planes_last, sh.fp16,
                                              sh.pscale_r, dbg);
    };
    for (int l0 = 0; l0 < sh.m; l0 += 32) {
        const int mm = sh.m - l0 < 32 ? sh.m - l0 : 32;   // R_l of this launch
        switch ((mm + 3) / 4) {
            case 1: go(k_contract_f32<4>, 4, l0); break;
            case 2: go(k_contract_f32<8>, 8, l0); break;
            case 3: go(k_contract_f32<12>, 12, l0); break;
            case 4: go(k_contract_f32<16>, 16, l0); break;
            case 5: go(k_contract_f32<20>, 20, l0); break;
            case 6: go(k_contract_f32<24>, 24, l0); break;
            case 7: go(k_contract_f32<28>, 28, l0); break;
            default: go(k_contract_f32<32>, 32, l0); break;
        }
    }
    if (planes_last > 0) k_mirror_planes<<<wsym.total, 256, 0, s>>>(in, wsym, sh.n_tslots, sh.m, planes_last,
                                                         sh.ublk, dbg);
    return cudaGetLastError();
}

}  // namespace fo
