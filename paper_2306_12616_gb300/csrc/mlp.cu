// Learned chemical potential: features, the network (forward, backward, Adam), the
// proposal of mu and the trace judge with its corrections.
//
// The paper fixes mu by hand. Here a small fully connected network (68 -> 256 -> 256 -> 2,
// SiLU, float32) maps the moments tau_1..tau_64 / N that the baby steps already give (plus
// N_e / N, kT on the scaled axis and the bounds) to mu on the scaled axis and to the order
// of the expansion; it is trained on (H, mu) pairs the exact method generates. A proposed
// mu is only kept when the float64 trace of the resulting P meets the tolerance; otherwise
// mu is corrected from tr P and ||P||_F^2 (Newton, then secant) and P re-evaluated, and
// instances that still miss fall back to exact moments and bisection.
//
// Every reduction runs in a fixed order (one thread per output, sequential sums), so
// training and inference are deterministic.
#include "internal.cuh"

namespace fo {
namespace {

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z) {
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// out[b, o] = act(sum_i in[b, i] W[o, i] + bias[o]); z[b, o] = the pre-activation.
__global__ void k_dense_fwd(const float* __restrict__ in, int B, int I, const float* __restrict__ W,
                            const float* __restrict__ bias, int O, int act, float* __restrict__ z,
                            float* __restrict__ out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (o >= O || b >= B) return;
    const float* x = in + (int64_t)b * I;
    const float* w = W + (int64_t)o * I;
    float s = bias[o];
    for (int i = 0; i < I; ++i) s = fmaf(x[i], w[i], s);
    if (z) z[(int64_t)b * O + o] = s;
    out[(int64_t)b * O + o] = act ? silu_f(s) : s;
}

// dW[o, i] = sum_b dZ[b, o] A[b, i]; db[o] = sum_b dZ[b, o] (thread (o, I) does the bias).
__global__ void k_dense_bwd_w(const float* __restrict__ dZ, const float* __restrict__ A, int B, int I, int O,
                              float* __restrict__ dW, float* __restrict__ db) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, o = blockIdx.y;
    if (i > I || o >= O) return;
    float s = 0.0f;
    if (i < I) {
        for (int b = 0; b < B; ++b) s = fmaf(dZ[(int64_t)b * O + o], A[(int64_t)b * I + i], s);
        dW[(int64_t)o * I + i] = s;
    } else {
        for (int b = 0; b < B; ++b) s += dZ[(int64_t)b * O + o];
        db[o] = s;
    }
}

// dZprev[b, i] = (sum_o dZ[b, o] W[o, i]) silu'(zprev[b, i]).
__global__ void k_dense_bwd_x(const float* __restrict__ dZ, const float* __restrict__ W, int B, int I, int O,
                              const float* __restrict__ zprev, float* __restrict__ dZprev) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (i >= I || b >= B) return;
    float s = 0.0f;
    for (int o = 0; o < O; ++o) s = fmaf(dZ[(int64_t)b * O + o], W[(int64_t)o * I + i], s);
    dZprev[(int64_t)b * I + i] = s * silu_grad_f(zprev[(int64_t)b * I + i]);
}

// Weighted squared error L = (1/B) sum_b sum_j w_j (y - t)^2 and dL/dy; one block.
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, int B, float w0, float w1,
                      float* __restrict__ dy, float* __restrict__ loss) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int q = threadIdx.x; q < 2 * B; q += blockDim.x) {
        const float w = (q & 1) ? w1 : w0;
        const float d = y[q] - t[q];
        dy[q] = 2.0f * w * d / (float)B;
        s += (double)w * d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
        *loss = (float)(tot / B);
    }
}

// Adam (Kingma and Ba) with bias-corrected moments; step counts from 1.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, int step) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float mq = b1 * m[q] + (1.0f - b1) * g[q];
    const float vq = b2 * v[q] + (1.0f - b2) * g[q] * g[q];
    m[q] = mq;
    v[q] = vq;
    const float mh = mq / (1.0f - powf(b1, (float)step));
    const float vh = vq / (1.0f - powf(b2, (float)step));
    p[q] -= lr * mh / (sqrtf(vh) + eps);
}

// dst[r, :] = (src[idx[r], :] - mean) / std
__global__ void k_gather_norm(const float* __restrict__ src, const int* __restrict__ idx, int B, int C,
                              const float* __restrict__ mean, const float* __restrict__ stdv, float* __restrict__ dst) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (c >= C || r >= B) return;
    const int s = idx ? idx[r] : r;
    dst[(int64_t)r * C + c] = (src[(int64_t)s * C + c] - mean[c]) / stdv[c];
}

// Column mean and standard deviation (float64 sums in row order); std floored at 1e-6 of
// max(1, |mean|) so that constant columns map to zero. One block per column.
__global__ void k_col_stats(const float* __restrict__ X, int n, int C, float* __restrict__ mean,
                            float* __restrict__ stdv) {
    __shared__ double sh[2][32];
    const int c = blockIdx.x;
    double s = 0.0, q = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const double v = X[(int64_t)r * C + c];
        s += v;
        q += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = s; sh[1][threadIdx.x >> 5] = q; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tq = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { ts += sh[0][w]; tq += sh[1][w]; }
        const double mu = ts / n;
        const double var = fmax(tq / n - mu * mu, 0.0);
        mean[c] = (float)mu;
        stdv[c] = (float)fmax(sqrt(var), 1e-6 * fmax(1.0, fabs(mu)));
    }
}

// Features of every instance (row = caller index when rows_by_user, else plan order):
// tau_1..tau_64 / n (tau_j, j > 2k, zero), N_e / n, 2 kT / (e_b - e_a), e_a / 100, e_b / 100.
__global__ void k_features(const Inst* __restrict__ insts, const InstIO* __restrict__ io, int batch, int k,
                           int rows_by_user, float* __restrict__ feat) {
    const int i = blockIdx.x, c = threadIdx.x;
    if (i >= batch || c >= kMlpIn) return;
    const Inst& in = insts[i];
    const DevResult* r = in.res;
    const double n = (double)in.n;
    const double ea = r->bounds[0], eb = r->bounds[1];
    double v = 0.0;
    if (c < kMlpMoments) v = (c + 1 <= 2 * k) ? in.tau[c + 1] / n : 0.0;
    else if (c == kMlpMoments) v = io[i].n_e / n;
    else if (c == kMlpMoments + 1) v = 2.0 * io[i].kT / (eb - ea);
    else if (c == kMlpMoments + 2) v = ea / 100.0;
    else v = eb / 100.0;
    const int row = rows_by_user ? in.user : i;
    feat[(int64_t)row * kMlpIn + c] = (float)v;
}

// Targets (mu_x, log2(L*) / log2(n_terms)) of every instance, from its mu, bounds and
// coefficients c_j(mu) (L*: the smallest L with sum_{j >= L} |c_j| <= kOrderEps). Row =
// caller index.
__global__ void k_targets(const Inst* __restrict__ insts, int batch, int n_terms, float* __restrict__ tgt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    const Inst& in = insts[i];
    const DevResult* r = in.res;
    const double ea = r->bounds[0], eb = r->bounds[1];
    // the order target: the smallest L with sum_{j >= L} |c_j| <= kOrderEps, so that the
    // expansion cut at L terms is within kOrderEps of the full one in the 2-norm
    double tail = 0.0;
    int L = n_terms;
    for (int j = n_terms - 1; j >= 1; --j) {
        tail += fabs(in.c[j]);
        if (tail > kOrderEps) break;
        L = j;
    }
    const double lg = n_terms > 1 ? log2((double)n_terms) : 1.0;
    tgt[(int64_t)in.user * 2] = (float)((2.0 * r->mu - (ea + eb)) / (eb - ea));
    tgt[(int64_t)in.user * 2 + 1] = (float)(log2((double)(L > 1 ? L : 1)) / lg);
}

// Low moments tau_0..tau_{2k} from the baby-step traces diag[0..k) (T_1..T_k) and
// gram[i-1] = <T_k, T_i>, i = 1..k: tau_{k+i} = 2 <T_k, T_i> - tau_{k-i} (Eq. identity).
__global__ void k_assemble_low(const Inst* __restrict__ insts, int batch, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    const Inst& in = insts[i];
    if (!in.res->active) return;
    double* tau = in.tau;
    tau[0] = (double)in.n;
    for (int j = 1; j <= k; ++j) tau[j] = in.diag[j - 1];
    for (int j = 1; j <= k; ++j) tau[k + j] = 2.0 * in.gram[j - 1] - tau[k - j];
}

// mu0 = mid + half (m_x + s_x y0) clamped into the bounds, order = n_terms^(m_o + s_o y1).
// The network's proposals: mu, and the expansion order L* (the number of terms whose
// coefficient tail sum_{j >= L*} |c_j| is at most kOrderEps). With use_order the instance's expansion is cut at
// n_eff = k m_eff coefficients, m_eff = ceil(margin L* / k) giant steps, clamped to [2, m]:
// every coefficient from n_eff on is zero, and the products whose outputs that leaves zero
// or unused are skipped (step_needed).
__global__ void k_learned_mu(const Inst* __restrict__ insts, int batch, const float* __restrict__ y,
                             const float* __restrict__ norm, int n_terms, int k, int m, int use_order,
                             double margin) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    DevResult* r = insts[i].res;
    const double ea = r->bounds[0], eb = r->bounds[1];
    const float* tmean = norm + 2 * kMlpIn;
    const float* tstd = tmean + kMlpOut;
    const double mx = (double)tmean[0] + (double)tstd[0] * (double)y[2 * i];
    const double lo = (double)tmean[1] + (double)tstd[1] * (double)y[2 * i + 1];
    double mu = 0.5 * (ea + eb) + 0.5 * (eb - ea) * mx;
    mu = fmin(fmax(mu, ea), eb);
    r->mu = r->mu0 = mu;
    r->order = exp2(lo * log2((double)(n_terms > 1 ? n_terms : 2)));
    if (use_order && m >= 2 && isfinite(r->order)) {
        int me = (int)ceil(margin * fmax(r->order, 1.0) / (double)k);
        me = me < 2 ? 2 : (me > m ? m : me);
        r->m_eff = me;
        r->n_eff = k * me < n_terms ? k * me : n_terms;
    }
}

// The judge after evaluation `round` (0 = at the learned mu): accept when |tr P - N_e| <=
// tol (tol <= 0: 1e-8 max(1, N_e) for float64, 1e-7 n for the split forms); otherwise, if
// rounds remain, move mu by a Newton step on d tr P / d mu ~ tr(P (I - P)) / kT_p =
// (tr P - ||P||_F^2) / kT_p (first round; kT_p the effective temperature of the truncated
// expansion, k_poly_width, which is kT for an exact Fermi function) or a secant step
// through the previous evaluation, limited to 10 kT_p; else leave the instance active for
// the bisection fallback.
__global__ void k_learned_check(const Inst* __restrict__ insts, const InstIO* __restrict__ io, int batch,
                                int round, int max_rounds, double tol, int is64, int* __restrict__ active_count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    DevResult* r = insts[i].res;
    if (!r->active) return;
    const double n_e = io[i].n_e, kT = io[i].kT;
    // default: float64 meets the strict trace bar; the split forms are judged within the band
    // of their float32 rounding of tr P (the trace correction then removes that part)
    const double t = tol > 0.0 ? tol : (is64 ? 1e-8 * fmax(1.0, n_e) : 1e-7 * (double)insts[i].n);
    const double err = r->trace - n_e;
    r->evals = round + 1;
    if (fabs(err) <= t && isfinite(err)) {
        r->active = 0;
        r->learned_ok = 1;
        return;
    }
    if (round >= max_rounds) {
        r->learned_ok = 0;   // stays active: exact moments and bisection follow
        atomicAdd(active_count, 1);
        return;
    }
    const double kte = (r->kt_eff > 0.0 && isfinite(r->kt_eff)) ? fmax(r->kt_eff, kT) : kT;
    double slope = (r->trace - r->frob2) / kte;
    if (round > 0 && r->mu != r->mu_prev) {
        const double sec = (r->trace - r->tr_prev) / (r->mu - r->mu_prev);
        if (sec > 0.0 && isfinite(sec)) slope = sec;
    }
    double step = (slope > 0.0 && isfinite(slope)) ? -err / slope : 0.0;
    step = fmin(fmax(step, -10.0 * kte), 10.0 * kte);
    r->mu_prev = r->mu;
    r->tr_prev = r->trace;
    r->mu = r->mu + step;
    atomicAdd(active_count, 1);
}

}  // namespace

// ------------------------------------------------------------------ launchers
cudaError_t mlp_forward(const float* params, const float* x, int B, float* z1, float* a1, float* z2, float* a2,
                        float* y, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    const MlpOffsets o = mlp_offsets();
    k_dense_fwd<<<dim3((kMlpHidden + 127) / 128, B), 128, 0, s>>>(x, B, kMlpIn, params + o.W1, params + o.b1,
                                                                  kMlpHidden, 1, z1, a1);
    k_dense_fwd<<<dim3((kMlpHidden + 127) / 128, B), 128, 0, s>>>(a1, B, kMlpHidden, params + o.W2, params + o.b2,
                                                                  kMlpHidden, 1, z2, a2);
    k_dense_fwd<<<dim3(1, B), 32, 0, s>>>(a2, B, kMlpHidden, params + o.W3, params + o.b3, kMlpOut, 0, nullptr, y);
    return cudaGetLastError();
}

cudaError_t mlp_backward(const float* params, const float* x, const float* t, int B, const float* z1,
                         const float* a1, const float* z2, const float* a2, const float* y, float* dy, float* dz2,
                         float* dz1, float* grad, float* loss, cudaStream_t s) {
    const MlpOffsets o = mlp_offsets();
    k_mse<<<1, 256, 0, s>>>(y, t, B, kMlpLossW0, kMlpLossW1, dy, loss);
    k_dense_bwd_w<<<dim3((kMlpHidden + 1 + 127) / 128, kMlpOut), 128, 0, s>>>(dy, a2, B, kMlpHidden, kMlpOut,
                                                                              grad + o.W3, grad + o.b3);
    k_dense_bwd_x<<<dim3((kMlpHidden + 127) / 128, B), 128, 0, s>>>(dy, params + o.W3, B, kMlpHidden, kMlpOut,
                                                                    z2, dz2);
    k_dense_bwd_w<<<dim3((kMlpHidden + 1 + 127) / 128, kMlpHidden), 128, 0, s>>>(dz2, a1, B, kMlpHidden,
                                                                                 kMlpHidden, grad + o.W2,
                                                                                 grad + o.b2);
    k_dense_bwd_x<<<dim3((kMlpHidden + 127) / 128, B), 128, 0, s>>>(dz2, params + o.W2, B, kMlpHidden,
                                                                    kMlpHidden, z1, dz1);
    k_dense_bwd_w<<<dim3((kMlpIn + 1 + 127) / 128, kMlpHidden), 128, 0, s>>>(dz1, x, B, kMlpIn, kMlpHidden,
                                                                             grad + o.W1, grad + o.b1);
    return cudaGetLastError();
}

cudaError_t mlp_adam(float* p, const float* g, float* m, float* v, int n, float lr, int step, cudaStream_t s) {
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(p, g, m, v, n, lr, 0.9f, 0.999f, 1e-8f, step);
    return cudaGetLastError();
}

cudaError_t mlp_gather_norm(const float* src, const int* idx, int B, int C, const float* mean, const float* stdv,
                            float* dst, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    k_gather_norm<<<dim3((C + 127) / 128, B), 128, 0, s>>>(src, idx, B, C, mean, stdv, dst);
    return cudaGetLastError();
}

cudaError_t mlp_col_stats(const float* X, int n, int C, float* mean, float* stdv, cudaStream_t s) {
    k_col_stats<<<C, 256, 0, s>>>(X, n, C, mean, stdv);
    return cudaGetLastError();
}

cudaError_t launch_features(const Inst* in, const InstIO* io, int batch, int k, int rows_by_user, float* feat,
                            cudaStream_t s) {
    k_features<<<batch, 96, 0, s>>>(in, io, batch, k, rows_by_user, feat);
    return cudaGetLastError();
}

cudaError_t launch_targets(const Inst* in, int batch, int n_terms, float* tgt, cudaStream_t s) {
    k_targets<<<(batch + 127) / 128, 128, 0, s>>>(in, batch, n_terms, tgt);
    return cudaGetLastError();
}

cudaError_t launch_assemble_low(const Inst* in, int batch, int k, cudaStream_t s) {
    k_assemble_low<<<(batch + 127) / 128, 128, 0, s>>>(in, batch, k);
    return cudaGetLastError();
}

cudaError_t launch_learned_mu(const Inst* in, int batch, const float* y, const float* norm, int n_terms,
                              int k, int m, int use_order, double margin, cudaStream_t s) {
    k_learned_mu<<<(batch + 127) / 128, 128, 0, s>>>(in, batch, y, norm, n_terms, k, m, use_order, margin);
    return cudaGetLastError();
}

cudaError_t launch_learned_check(const Inst* in, const InstIO* io, int batch, int round, int max_rounds,
                                 double tol, int is64, int* active_count, cudaStream_t s) {
    k_learned_check<<<(batch + 127) / 128, 128, 0, s>>>(in, io, batch, round, max_rounds, tol, is64, active_count);
    return cudaGetLastError();
}

}  // namespace fo
