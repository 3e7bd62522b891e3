// Internal declarations shared by the CUDA translation units of the solver.
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

// Device-resident record of the scalar results of one density-matrix evaluation.
struct DevResult {
    double bounds[2];     // emin, emax
    double mu;
    double trace;         // tr P
    double frob2;         // ||P||_F^2
    double trace_poly;    // sum_n c_n tau_n at mu
    int32_t iters;        // bisection halvings
    int32_t status;       // fo_status of device stages
    int32_t nonfinite;    // H held NaN/Inf
    int32_t learned_ok;   // learned mu accepted
    int32_t tc_timeout;   // a tensor-core kernel gave up a bounded wait
    int32_t pad_;
    double mu_lo, mu_hi;  // final bisection bracket
};

// A float32 working matrix with its 16-bit split planes (plane p at planes + p*plane_stride).
struct MatF32 {
    float* x;
    uint16_t* planes;
    int64_t ld;
    int64_t plane_stride;  // elements
};

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

// Epilogue of one recurrence product: out = alpha*acc + beta*C + D + shift*I_{n_real}.
struct Epilogue {
    float alpha, beta, shift;
    int32_t n_real;                // identity and output rows/cols limited to this
    const float* C;                // float32 masters, leading dimension ld (may be null)
    const float* D;
    int64_t ld;
    MatF32 out;                    // slot output (x may be null when writing out64)
    double* out64;                 // final float64 output (user buffer), or null
    int64_t ldo;
    int32_t planes;                // 16-bit planes to write for `out` (0..3)
    int32_t fp16;                  // planes are fp16 (else bf16)
    float plane_scale;             // value multiplied into the planes before splitting
    int* dbg;                      // self-check record (null unless built with FO_SELF_CHECK)
};

// Split/packing helpers (reduce.cu)
cudaError_t launch_gershgorin(const double* H, int64_t n, int64_t ld, double* part_lo,
                              double* part_hi, int* part_bad, int nparts, DevResult* res,
                              int use_given, double emin, double emax, cudaStream_t s);
cudaError_t launch_set_bounds(DevResult* res, double emin, double emax, cudaStream_t s);
cudaError_t launch_set_scalar(double* dst, double v, cudaStream_t s);
cudaError_t launch_export_bounds(const DevResult* res, double* out3, cudaStream_t s);
cudaError_t launch_scale_f64(const double* H, int64_t n, int64_t ld, const DevResult* res,
                             double* X, int64_t np, cudaStream_t s, int* dbg);
cudaError_t launch_scale_split(const double* H, int64_t n, int64_t ld, const DevResult* res,
                               MatF32 X, int64_t np, int planes, int fp16, float pscale,
                               cudaStream_t s, int* dbg);
cudaError_t launch_pack_f32(const float* A, int64_t n, int64_t lda, MatF32 X, int64_t np,
                            int planes, int fp16, float pscale, cudaStream_t s);
cudaError_t launch_diag_sums(const void* base, int64_t slot_stride_bytes, int count,
                             int64_t n, int64_t np, int is_f64, double* out, cudaStream_t s);
cudaError_t launch_gram(const void* base, int64_t slot_stride_bytes, int giant0, int ngiant,
                        int baby0, int nbaby, int64_t np, int is_f64, double* partials,
                        int max_blocks, double* out, cudaStream_t s);
int gram_blocks(int64_t np, int ngiant, int nbaby);
cudaError_t launch_assemble_moments(const double* diag, const double* gram, int k, int m,
                                    int n_terms, int64_t n, double* tau, cudaStream_t s);
cudaError_t launch_trace_frob(const double* P, int64_t n, int64_t ldp, double* partials,
                              int nparts, DevResult* res, cudaStream_t s);
cudaError_t launch_copy_out(const double* R, int64_t np, int64_t n, double* P, int64_t ldp,
                            cudaStream_t s);
cudaError_t launch_copy_out_f32(const float* R, int64_t np, int64_t n, double* P, int64_t ldp,
                                cudaStream_t s);

// Coefficient pipeline (coef.cu)
cudaError_t launch_cos_table(int M, double* ct, cudaStream_t s);
cudaError_t launch_dos_weights(const double* tau, int n_terms, int M, const double* ct,
                               double* w, cudaStream_t s);
cudaError_t launch_bisect(const double* w, const double* ct, int M, DevResult* res, double kT,
                          double n_e, int max_iter, cudaStream_t s);
cudaError_t launch_fermi_nodes(int M, const double* ct, const DevResult* res, double kT,
                               double* f, cudaStream_t s);
cudaError_t launch_coeffs(const double* f, const double* ct, int M, int n_terms, int km,
                          double* c, cudaStream_t s);
cudaError_t launch_g_convert(const double* c, int k, int m, double* g, cudaStream_t s);
cudaError_t launch_poly_trace(const double* c, const double* tau, int n_terms, DevResult* res,
                              cudaStream_t s);
cudaError_t launch_contract_f64(const double* g, int k, int m, const double* tbase,
                                int64_t tstride, double* rbase, int64_t rstride, int64_t n,
                                int64_t np, cudaStream_t s);
cudaError_t launch_contract_f32(const double* g, int k, int m, const float* tbase,
                                int64_t tstride_f, float* rbase, int64_t rstride_f, int64_t n,
                                int64_t np, int planes_last, int fp16, float pscale,
                                int64_t plane_off_f, cudaStream_t s, int* dbg);

// Matrix products (gemm_f64.cu, gemm_tc.cu)
// out = alpha*A*B + beta*C + D + shift*I_{n_real}; all np x np float64 with ld np. Only
// the tiles on or above the diagonal are computed; each is written at (r,c) and (c,r).
// If out64 != null the result goes to out64[n_real x n_real, ldo] instead of out.
cudaError_t launch_gemm_f64(const double* A, const double* B, int64_t np, double alpha,
                            const double* C, double beta, const double* D, double shift,
                            int n_real, double* out, double* out64, int64_t ldo,
                            cudaStream_t s);

// Tensor-core split-precision product. A, B are slots (float32 master + planes). B is read
// transposed (B^T), which equals B for the exactly symmetric matrices of the method. With
// sym != 0 only the tiles on or above the diagonal are computed and mirrored.
cudaError_t tc_gemm(int prec, int64_t np, const MatF32& A, const MatF32& B, const Epilogue& ep,
                    int sym, int* err_flag, cudaStream_t s, std::string* err);
int64_t tc_tiles(int64_t np, int sym);
int tc_planes(int prec);

}  // namespace fo
