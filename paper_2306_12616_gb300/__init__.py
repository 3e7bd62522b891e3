"""Python binding of the GB300 dense Chebyshev Fermi-operator solver (include/fermi.h).

The functions named ``fo_*`` mirror the C ABI one to one: they only marshal arguments
(integers for device pointers and streams, ctypes structures for parameters) and call the
shared library built from csrc/. Every step of the method runs in the library's CUDA
kernels. There is no fallback: if the library has not been built, or no CUDA device is
present, the calls raise.

``Solver`` is a convenience wrapper over the same calls for torch tensors.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

__all__ = [
    "FO_OK", "FO_PREC_FP64", "FO_PREC_BF16X3", "FO_PREC_FP16X2", "FO_PREC_BF16X1",
    "FO_MU_FIXED", "FO_MU_BISECT", "FO_MU_LEARNED", "FO_MU_ORDER", "FO_FLAG_NO_RESULT_SYNC", "FO_FLAG_GRAPH",
    "FO_FLAG_STAGED", "FO_FLAG_POWER_BASIS", "FO_FLAG_NO_TRACE_FIX", "FO_FLAG_ALLOW_LOOSE",
    "FoParams", "FoResult", "FermiError", "lib", "library_path", "EXPORTED_SYMBOLS",
    "fo_create", "fo_destroy", "fo_last_error", "fo_status_string", "fo_version",
    "fo_spectral_bounds", "fo_chebyshev_coeffs", "fo_density_matrix", "fo_density_matrix_host",
    "fo_density_matrix_batched", "fo_density_matrix_batched_host", "fo_host_wait", "fo_moments",
    "fo_recurrence_product", "fo_profile_enable", "fo_profile_read", "FoProfile",
    "fo_spectral_bounds_noalloc", "FO_NOALLOC_MAX_N", "fo_learned_features", "fo_mlp_init",
    "fo_mlp_set_params", "fo_mlp_get_params", "fo_mlp_forward", "fo_mlp_gradients", "fo_mlp_train",
    "fo_mlp_save", "fo_mlp_load", "FO_MLP_INPUTS", "FO_MLP_OUTPUTS", "FO_MLP_PARAMS", "FO_MLP_NORM",
    "STAGE_NAMES", "Solver", "PRECISIONS", "MU_MODES",
]

FO_OK = 0
FO_ERR_ARG, FO_ERR_CUDA, FO_ERR_NOMEM, FO_ERR_NONFINITE = 1, 2, 3, 4
FO_ERR_NO_BRACKET, FO_ERR_NOT_CONVERGED, FO_ERR_DEVICE_TIMEOUT, FO_ERR_UNSUPPORTED = 5, 6, 7, 8
FO_PREC_FP64, FO_PREC_BF16X3, FO_PREC_FP16X2, FO_PREC_BF16X1 = 0, 1, 2, 3
FO_MU_FIXED, FO_MU_BISECT, FO_MU_LEARNED, FO_MU_ORDER = 0, 1, 2, 3
FO_FLAG_NO_RESULT_SYNC = 0x2
FO_FLAG_GRAPH = 0x4
FO_FLAG_STAGED = 0x8
FO_FLAG_POWER_BASIS = 0x10
FO_FLAG_NO_TRACE_FIX = 0x20
FO_FLAG_ALLOW_LOOSE = 0x40

PRECISIONS = {"fp64": FO_PREC_FP64, "bf16x3": FO_PREC_BF16X3, "fp16x2": FO_PREC_FP16X2,
              "bf16x1": FO_PREC_BF16X1}
MU_MODES = {"fixed": FO_MU_FIXED, "bisect": FO_MU_BISECT, "learned": FO_MU_LEARNED, "order": FO_MU_ORDER}

# Every symbol the header declares (checked by the CPU test suite against the .so).
EXPORTED_SYMBOLS = (
    "fo_create", "fo_destroy", "fo_last_error", "fo_status_string", "fo_version",
    "fo_spectral_bounds", "fo_spectral_bounds_noalloc", "fo_chebyshev_coeffs", "fo_density_matrix",
    "fo_density_matrix_host", "fo_density_matrix_batched", "fo_density_matrix_batched_host", "fo_host_wait",
    "fo_moments", "fo_recurrence_product", "fo_profile_enable", "fo_profile_read", "fo_learned_features", "fo_mlp_init",
    "fo_mlp_set_params", "fo_mlp_get_params", "fo_mlp_forward", "fo_mlp_gradients", "fo_mlp_train",
    "fo_mlp_save", "fo_mlp_load",
)
FO_NOALLOC_MAX_N = 32768
FO_MLP_INPUTS, FO_MLP_OUTPUTS, FO_MLP_PARAMS, FO_MLP_NORM = 68, 2, 83970, 140


class FoParams(ctypes.Structure):
    _fields_ = [
        ("n_terms", ctypes.c_int32), ("k", ctypes.c_int32), ("kT", ctypes.c_double),
        ("mu", ctypes.c_double), ("precision", ctypes.c_int32), ("mu_mode", ctypes.c_int32),
        ("use_given_bounds", ctypes.c_int32), ("n_quad", ctypes.c_int32),
        ("emin", ctypes.c_double), ("emax", ctypes.c_double), ("max_bisect", ctypes.c_int32),
        ("flags", ctypes.c_uint32), ("tr_tol", ctypes.c_double), ("max_newton", ctypes.c_int32),
        ("tile_n", ctypes.c_int32), ("tile_ctas", ctypes.c_int32), ("lanczos_steps", ctypes.c_int32),
        ("tile_drain", ctypes.c_int32), ("tile_store", ctypes.c_int32), ("chain", ctypes.c_int32),
        ("tile_persist", ctypes.c_int32), ("chain_window", ctypes.c_int32),
    ]


class FoResult(ctypes.Structure):
    _fields_ = [
        ("mu", ctypes.c_double), ("trace", ctypes.c_double), ("trace_poly", ctypes.c_double),
        ("frob2", ctypes.c_double), ("emin", ctypes.c_double), ("emax", ctypes.c_double),
        ("k", ctypes.c_int32), ("m", ctypes.c_int32), ("n_gemm", ctypes.c_int32),
        ("bisect_iters", ctypes.c_int32), ("learned_accepted", ctypes.c_int32),
        ("status", ctypes.c_int32), ("n_launches", ctypes.c_int32), ("tile_n", ctypes.c_int32),
        ("tile_ctas", ctypes.c_int32), ("evals", ctypes.c_int32), ("order", ctypes.c_int32),
        ("tile_drain", ctypes.c_int32), ("tile_store", ctypes.c_int32),
        ("trace_raw", ctypes.c_double), ("trace_gamma", ctypes.c_double), ("trace_proj", ctypes.c_double),
        ("tile_persist", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


FO_PROFILE_STAGES = 8
STAGE_NAMES = ("bounds", "products", "moments", "mu", "coeffs", "contract", "trace", "call")


class FoProfile(ctypes.Structure):
    _fields_ = [
        ("ms", ctypes.c_double * FO_PROFILE_STAGES),
        ("flops", ctypes.c_double * FO_PROFILE_STAGES),
        ("launches", ctypes.c_int64 * FO_PROFILE_STAGES),
        ("calls", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {name: {"ms": self.ms[i], "flops": self.flops[i], "launches": self.launches[i]}
                for i, name in enumerate(STAGE_NAMES)} | {"calls": self.calls}


class FermiError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


def library_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libfermi_gb300.so")


_LIB = None
_c_ptr, _c_i64, _c_i32, _c_d, _c_f = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_float)


def lib() -> ctypes.CDLL:
    """Load the shared library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run paper_2306_12616_gb300/build.py)")
        L = ctypes.CDLL(path)
        sig = {
            "fo_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]),
            "fo_destroy": (ctypes.c_int, [_c_ptr]),
            "fo_last_error": (ctypes.c_char_p, [_c_ptr]),
            "fo_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "fo_version": (ctypes.c_char_p, []),
            "fo_spectral_bounds": (ctypes.c_int, [_c_ptr, _c_ptr, _c_i64, _c_i64, _c_ptr, _c_ptr]),
            "fo_chebyshev_coeffs": (ctypes.c_int, [_c_ptr, _c_d, _c_d, _c_d, _c_d, _c_i32, _c_i32,
                                                   _c_ptr, _c_ptr]),
            "fo_density_matrix": (ctypes.c_int, [_c_ptr, _c_ptr, _c_i64, _c_i64, _c_d,
                                                 ctypes.POINTER(FoParams), _c_ptr, _c_i64,
                                                 ctypes.POINTER(FoResult), _c_ptr]),
            "fo_density_matrix_host": (ctypes.c_int, [_c_ptr, _c_ptr, _c_i64, _c_i64, _c_d,
                                                      ctypes.POINTER(FoParams), _c_ptr, _c_i64,
                                                      ctypes.POINTER(FoResult), _c_ptr]),
            "fo_density_matrix_batched": (ctypes.c_int, [_c_ptr, _c_i32, _c_ptr, _c_ptr, _c_ptr, _c_ptr,
                                                         _c_ptr, ctypes.POINTER(FoParams), _c_ptr, _c_ptr,
                                                         _c_ptr, _c_ptr]),
            "fo_density_matrix_batched_host": (ctypes.c_int, [_c_ptr, _c_i32, _c_ptr, _c_ptr, _c_ptr, _c_ptr,
                                                              _c_ptr, ctypes.POINTER(FoParams), _c_ptr,
                                                              _c_ptr, _c_ptr, _c_ptr]),
            "fo_host_wait": (ctypes.c_int, [_c_ptr]),
            "fo_learned_features": (ctypes.c_int, [_c_ptr, _c_i32, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr,
                                                   ctypes.POINTER(FoParams), _c_ptr, _c_ptr, _c_ptr, _c_ptr]),
            "fo_mlp_init": (ctypes.c_int, [_c_ptr, ctypes.c_uint64]),
            "fo_mlp_set_params": (ctypes.c_int, [_c_ptr, _c_ptr, _c_ptr]),
            "fo_mlp_get_params": (ctypes.c_int, [_c_ptr, _c_ptr, _c_ptr]),
            "fo_mlp_forward": (ctypes.c_int, [_c_ptr, _c_ptr, _c_i32, _c_ptr, _c_ptr]),
            "fo_mlp_gradients": (ctypes.c_int, [_c_ptr, _c_ptr, _c_ptr, _c_i32, _c_ptr, _c_ptr, _c_ptr]),
            "fo_mlp_train": (ctypes.c_int, [_c_ptr, _c_ptr, _c_ptr, _c_i32, _c_i32, _c_i32, _c_f,
                                            ctypes.c_uint64, _c_ptr, _c_ptr]),
            "fo_mlp_save": (ctypes.c_int, [_c_ptr, ctypes.c_char_p]),
            "fo_mlp_load": (ctypes.c_int, [_c_ptr, ctypes.c_char_p]),
            "fo_moments": (ctypes.c_int, [_c_ptr, _c_ptr, _c_i64, _c_i64, _c_ptr, _c_i32, _c_i32,
                                          _c_ptr, _c_ptr]),
            "fo_profile_enable": (ctypes.c_int, [_c_ptr, _c_i32]),
            "fo_spectral_bounds_noalloc": (ctypes.c_int, [_c_ptr, _c_i64, _c_i64, _c_ptr, _c_ptr]),
            "fo_profile_read": (ctypes.c_int, [_c_ptr, ctypes.POINTER(FoProfile), _c_i32]),
            "fo_recurrence_product": (ctypes.c_int, [_c_ptr, _c_i32, _c_i32, _c_i64, _c_i64, _c_ptr, _c_ptr,
                                                     _c_ptr, _c_ptr, _c_f, _c_f, _c_f, _c_ptr,
                                                     _c_ptr]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


# ----------------------------------------------------------------- C ABI, one to one

def fo_create(device: int = 0) -> int:
    h = ctypes.c_void_p()
    st = lib().fo_create(ctypes.byref(h), device)
    if st != FO_OK:
        raise FermiError(st, f"fo_create failed: {fo_status_string(st)}")
    return h.value


def fo_destroy(ctx: int) -> int:
    return lib().fo_destroy(ctx)


def fo_last_error(ctx: int) -> str:
    return lib().fo_last_error(ctx).decode()


def fo_status_string(status: int) -> str:
    return lib().fo_status_string(status).decode()


def fo_version() -> str:
    return lib().fo_version().decode()


def fo_spectral_bounds(ctx, d_h, n, ld, d_bounds, stream=0) -> int:
    return lib().fo_spectral_bounds(ctx, d_h, n, ld, d_bounds, stream)


def fo_spectral_bounds_noalloc(d_h, n, ld, d_bounds, stream=0) -> int:
    """Spectral bounds without a context or any device allocation (see include/fermi.h)."""
    return lib().fo_spectral_bounds_noalloc(d_h, n, ld, d_bounds, stream)


def fo_chebyshev_coeffs(ctx, kT, mu, emin, emax, n_terms, n_quad, d_c, stream=0) -> int:
    return lib().fo_chebyshev_coeffs(ctx, kT, mu, emin, emax, n_terms, n_quad, d_c, stream)


def fo_density_matrix(ctx, d_h, n, ld, n_e, params: FoParams, d_p, ldp, result: FoResult | None,
                      stream=0) -> int:
    return lib().fo_density_matrix(ctx, d_h, n, ld, n_e, ctypes.byref(params), d_p, ldp,
                                   ctypes.byref(result) if result is not None else None, stream)


def fo_density_matrix_host(ctx, h_h, n, ld, n_e, params: FoParams, h_p, ldp,
                           result: FoResult | None, stream=0) -> int:
    return lib().fo_density_matrix_host(ctx, h_h, n, ld, n_e, ctypes.byref(params), h_p, ldp,
                                        ctypes.byref(result) if result is not None else None,
                                        stream)


def fo_density_matrix_batched(ctx, batch, d_h_ptrs, n, ld, n_e, kT, params: FoParams, d_p_ptrs,
                              ldp, results, stream=0) -> int:
    """Arrays are ctypes arrays (or None where the header allows NULL); results is a ctypes
    array of FoResult of length batch, or None."""
    return lib().fo_density_matrix_batched(ctx, batch, d_h_ptrs, n, ld, n_e, kT, ctypes.byref(params),
                                           d_p_ptrs, ldp, results, stream)


def fo_density_matrix_batched_host(ctx, batch, h_h_ptrs, n, ld, n_e, kT, params: FoParams, h_p_ptrs,
                                   ldp, results, stream=0) -> int:
    return lib().fo_density_matrix_batched_host(ctx, batch, h_h_ptrs, n, ld, n_e, kT, ctypes.byref(params),
                                                h_p_ptrs, ldp, results, stream)


def fo_host_wait(ctx) -> int:
    return lib().fo_host_wait(ctx)


def fo_learned_features(ctx, batch, d_h_ptrs, n, ld, n_e, kT, params: FoParams, d_feat, d_target,
                        results, stream=0) -> int:
    return lib().fo_learned_features(ctx, batch, d_h_ptrs, n, ld, n_e, kT, ctypes.byref(params), d_feat,
                                     d_target, results, stream)


def fo_mlp_init(ctx, seed) -> int:
    return lib().fo_mlp_init(ctx, seed)


def fo_mlp_set_params(ctx, h_params, h_norm) -> int:
    return lib().fo_mlp_set_params(ctx, h_params, h_norm)


def fo_mlp_get_params(ctx, h_params, h_norm) -> int:
    return lib().fo_mlp_get_params(ctx, h_params, h_norm)


def fo_mlp_forward(ctx, d_x, n, d_y, stream=0) -> int:
    return lib().fo_mlp_forward(ctx, d_x, n, d_y, stream)


def fo_mlp_gradients(ctx, d_x, d_t, n, d_grad, h_loss, stream=0) -> int:
    return lib().fo_mlp_gradients(ctx, d_x, d_t, n, d_grad, h_loss, stream)


def fo_mlp_train(ctx, d_feat, d_target, n, epochs, batch, lr, seed, h_loss, stream=0) -> int:
    return lib().fo_mlp_train(ctx, d_feat, d_target, n, epochs, batch, lr, seed, h_loss, stream)


def fo_mlp_save(ctx, path: str) -> int:
    return lib().fo_mlp_save(ctx, path.encode())


def fo_mlp_load(ctx, path: str) -> int:
    return lib().fo_mlp_load(ctx, path.encode())


def fo_moments(ctx, d_h, n, ld, d_bounds, n_moments, precision, d_tau, stream=0) -> int:
    return lib().fo_moments(ctx, d_h, n, ld, d_bounds, n_moments, precision, d_tau, stream)


def fo_profile_enable(ctx, enable: int) -> int:
    return lib().fo_profile_enable(ctx, enable)


def fo_profile_read(ctx, profile: FoProfile, reset: int = 0) -> int:
    return lib().fo_profile_read(ctx, ctypes.byref(profile), reset)


def fo_recurrence_product(ctx, precision, symmetric, n, ld, d_a, d_b, d_c, d_d, alpha, beta,
                          shift, d_out, stream=0) -> int:
    return lib().fo_recurrence_product(ctx, precision, symmetric, n, ld, d_a, d_b, d_c, d_d, alpha,
                                       beta, shift, d_out, stream)


# ------------------------------------------------------------ torch convenience layer

def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


@dataclass
class Solver:
    """Owns one library context on a CUDA device; methods take torch tensors."""
    device: int = 0

    def __post_init__(self):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.ctx = fo_create(self.device)

    def close(self):
        if getattr(self, "ctx", None):
            fo_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != FO_OK:
            raise FermiError(st, fo_last_error(self.ctx) or fo_status_string(st))

    @staticmethod
    def params(n_terms: int, kT: float, *, mu: float = 0.0, precision: str | int = "fp64",
               mu_mode: str | int = "bisect", k: int = 0, bounds=None, n_quad: int = 0,
               max_bisect: int = 0, flags: int = 0, tile_n: int = 0, tile_ctas: int = 0,
               tr_tol: float = 0.0, max_newton: int = 0, lanczos_steps: int = 0,
               tile_drain: int = 0, tile_store: int = 0, chain: int = 0, chain_window: int = 0,
               tile_persist: int = 0) -> FoParams:
        p = FoParams()
        p.n_terms, p.k, p.kT, p.mu = n_terms, k, kT, mu
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
        p.mu_mode = MU_MODES[mu_mode] if isinstance(mu_mode, str) else mu_mode
        if bounds is not None:
            p.use_given_bounds, p.emin, p.emax = 1, float(bounds[0]), float(bounds[1])
        p.n_quad, p.max_bisect, p.flags = n_quad, max_bisect, flags
        p.tile_n, p.tile_ctas, p.tr_tol, p.max_newton = tile_n, tile_ctas, tr_tol, max_newton
        p.lanczos_steps, p.tile_drain, p.tile_store = lanczos_steps, tile_drain, tile_store
        p.chain, p.chain_window, p.tile_persist = chain, chain_window, tile_persist
        return p

    def spectral_bounds(self, h, stream=None):
        import torch
        out = torch.empty(3, dtype=torch.float64, device=h.device)
        self._check(fo_spectral_bounds(self.ctx, h.data_ptr(), h.shape[0], h.stride(0),
                                       out.data_ptr(), _stream_handle(stream)))
        return out

    def chebyshev_coeffs(self, kT, mu, emin, emax, n_terms, n_quad=0, stream=None):
        import torch
        out = torch.empty(n_terms, dtype=torch.float64, device=f"cuda:{self.device}")
        self._check(fo_chebyshev_coeffs(self.ctx, kT, mu, emin, emax, n_terms, n_quad,
                                        out.data_ptr(), _stream_handle(stream)))
        return out

    def density_matrix(self, h, n_e: float, params: FoParams, out=None, stream=None,
                       sync: bool = True):
        import torch
        assert h.dtype == torch.float64 and h.is_cuda and h.stride(1) == 1
        n = h.shape[0]
        p = out if out is not None else torch.empty((n, n), dtype=torch.float64, device=h.device)
        res = FoResult() if sync else None
        self._check(fo_density_matrix(self.ctx, h.data_ptr(), n, h.stride(0), float(n_e), params,
                                      p.data_ptr(), p.stride(0), res, _stream_handle(stream)))
        return p, (res.as_dict() if res is not None else None)

    def density_matrix_batched(self, hs, n_e, params: FoParams, kT=None, outs=None, stream=None,
                               sync: bool = True):
        """hs: list of CUDA float64 (n_b x n_b) tensors; n_e, kT: per-instance sequences
        (kT None: params.kT). Returns (list of P tensors, list of result dicts or None)."""
        import torch
        B = len(hs)
        for h in hs:
            assert h.dtype == torch.float64 and h.is_cuda and h.stride(1) == 1
        ps = outs if outs is not None else [torch.empty((h.shape[0], h.shape[0]), dtype=torch.float64,
                                                        device=h.device) for h in hs]
        ptr = ctypes.c_void_p * B
        i64 = ctypes.c_int64 * B
        dbl = ctypes.c_double * B
        d_h = ptr(*[h.data_ptr() for h in hs])
        d_p = ptr(*[p.data_ptr() for p in ps])
        n = i64(*[h.shape[0] for h in hs])
        ld = i64(*[h.stride(0) for h in hs])
        ldp = i64(*[p.stride(0) for p in ps])
        ne = dbl(*[float(x) for x in n_e])
        kt = dbl(*[float(x) for x in kT]) if kT is not None else None
        res = (FoResult * B)() if sync else None
        self._check(fo_density_matrix_batched(self.ctx, B, d_h, n, ld, ne, kt, params, d_p, ldp, res,
                                              _stream_handle(stream)))
        return ps, ([r.as_dict() for r in res] if res is not None else None)

    def density_matrix_batched_host(self, hs, n_e, params: FoParams, outs, kT=None, stream=None):
        """hs, outs: CPU float64 tensors (pinned for asynchronous copies). Returns result dicts;
        with FO_FLAG_NO_RESULT_SYNC in params the call only enqueues its copies and solve (the
        dicts are then not filled): keep hs unchanged and read outs after host_wait()."""
        B = len(hs)
        ptr, i64, dbl = ctypes.c_void_p * B, ctypes.c_int64 * B, ctypes.c_double * B
        res = (FoResult * B)()
        self._check(fo_density_matrix_batched_host(
            self.ctx, B, ptr(*[h.data_ptr() for h in hs]), i64(*[h.shape[0] for h in hs]),
            i64(*[h.stride(0) for h in hs]), dbl(*[float(x) for x in n_e]),
            dbl(*[float(x) for x in kT]) if kT is not None else None, params,
            ptr(*[o.data_ptr() for o in outs]), i64(*[o.stride(0) for o in outs]), res, _stream_handle(stream)))
        return [r.as_dict() for r in res]

    def host_wait(self):
        """Waits for every host-buffer call of this solver (fo_host_wait)."""
        self._check(fo_host_wait(self.ctx))

    # ------------------------------------------------------------ learned mu
    def learned_features(self, hs, n_e, params: FoParams, kT=None, stream=None):
        """Training pairs of a batch by the exact method: (features [B, 68], targets [B, 2],
        results) as float32 CUDA tensors and result dicts."""
        import torch
        B = len(hs)
        ptr, i64, dbl = ctypes.c_void_p * B, ctypes.c_int64 * B, ctypes.c_double * B
        feat = torch.empty((B, FO_MLP_INPUTS), dtype=torch.float32, device=hs[0].device)
        tgt = torch.empty((B, FO_MLP_OUTPUTS), dtype=torch.float32, device=hs[0].device)
        res = (FoResult * B)()
        self._check(fo_learned_features(
            self.ctx, B, ptr(*[h.data_ptr() for h in hs]), i64(*[h.shape[0] for h in hs]),
            i64(*[h.stride(0) for h in hs]), dbl(*[float(x) for x in n_e]),
            dbl(*[float(x) for x in kT]) if kT is not None else None, params, feat.data_ptr(), tgt.data_ptr(),
            res, _stream_handle(stream)))
        return feat, tgt, [r.as_dict() for r in res]

    def mlp_init(self, seed: int = 0):
        self._check(fo_mlp_init(self.ctx, seed))

    def mlp_set_params(self, params, norm=None):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == FO_MLP_PARAMS
        nrm = np.ascontiguousarray(norm, dtype=np.float32) if norm is not None else None
        self._check(fo_mlp_set_params(self.ctx, p.ctypes.data, nrm.ctypes.data if nrm is not None else None))

    def mlp_get_params(self):
        import numpy as np
        p = np.empty(FO_MLP_PARAMS, dtype=np.float32)
        nrm = np.empty(FO_MLP_NORM, dtype=np.float32)
        self._check(fo_mlp_get_params(self.ctx, p.ctypes.data, nrm.ctypes.data))
        return p, nrm

    def mlp_forward(self, x, stream=None):
        import torch
        y = torch.empty((x.shape[0], FO_MLP_OUTPUTS), dtype=torch.float32, device=x.device)
        self._check(fo_mlp_forward(self.ctx, x.data_ptr(), x.shape[0], y.data_ptr(), _stream_handle(stream)))
        return y

    def mlp_gradients(self, x, t, stream=None):
        import torch
        g = torch.empty(FO_MLP_PARAMS, dtype=torch.float32, device=x.device)
        loss = ctypes.c_float()
        self._check(fo_mlp_gradients(self.ctx, x.data_ptr(), t.data_ptr(), x.shape[0], g.data_ptr(),
                                     ctypes.byref(loss), _stream_handle(stream)))
        return g, loss.value

    def mlp_train(self, feat, target, epochs: int, batch: int = 256, lr: float = 1e-3, seed: int = 0,
                  stream=None):
        losses = (ctypes.c_float * epochs)()
        self._check(fo_mlp_train(self.ctx, feat.data_ptr(), target.data_ptr(), feat.shape[0], epochs, batch,
                                 lr, seed, losses, _stream_handle(stream)))
        return list(losses)

    def mlp_save(self, path: str):
        self._check(fo_mlp_save(self.ctx, path))

    def mlp_load(self, path: str):
        self._check(fo_mlp_load(self.ctx, path))

    def density_matrix_host(self, h, n_e: float, params: FoParams, out, stream=None):
        """h, out: CPU float64 tensors (pinned for asynchronous copies)."""
        res = FoResult()
        n = h.shape[0]
        self._check(fo_density_matrix_host(self.ctx, h.data_ptr(), n, h.stride(0), float(n_e),
                                           params, out.data_ptr(), out.stride(0), res,
                                           _stream_handle(stream)))
        return res.as_dict()

    def profile_enable(self, enable: bool = True):
        self._check(fo_profile_enable(self.ctx, 1 if enable else 0))

    def profile_read(self, reset: bool = False) -> dict:
        prof = FoProfile()
        self._check(fo_profile_read(self.ctx, prof, 1 if reset else 0))
        return prof.as_dict()

    def moments(self, h, bounds, n_moments: int, precision="fp64", stream=None):
        import torch
        tau = torch.empty(n_moments, dtype=torch.float64, device=h.device)
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        self._check(fo_moments(self.ctx, h.data_ptr(), h.shape[0], h.stride(0), bounds.data_ptr(),
                               n_moments, prec, tau.data_ptr(), _stream_handle(stream)))
        return tau

    def recurrence_product(self, a, b, c=None, d=None, alpha=1.0, beta=0.0, shift=0.0,
                           precision="bf16x3", symmetric=False, out=None, stream=None):
        import torch
        n = a.shape[0]
        o = out if out is not None else torch.empty_like(a)
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        self._check(fo_recurrence_product(
            self.ctx, prec, 1 if symmetric else 0, n, a.stride(0), a.data_ptr(), b.data_ptr(),
            c.data_ptr() if c is not None else None, d.data_ptr() if d is not None else None,
            alpha, beta, shift, o.data_ptr(), _stream_handle(stream)))
        return o
