"""ctypes binding of liblrq (C ABI in include/lrq.h).

Argument marshalling only: every function below has the name of the C entry
point it calls, takes torch tensors where the C function takes device
pointers, and raises LrqError when the call returns a non-zero lrq_status.
All computation happens in the CUDA kernels of liblrq.so; there is no
fallback -- if the library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblrq.so")

LRQ_OK = 0
LRQ_EINVAL = 1
LRQ_EUNSUPPORTED = 2
LRQ_ECUDA = 3
LRQ_ETIMEOUT = 4
LRQ_ENOCONV = 5
LRQ_EWORKSPACE = 6

LRQ_MODE_FP32 = 0
LRQ_MODE_TC = 1  # tensor-core mode: F16 x F16 (F16 accumulate) signs, FP8 E4M3 hi + lo class sums (FP32 accumulate)
LRQ_MODE_BF16_TC = LRQ_MODE_TC  # deprecated alias (the mode's first version used BF16 operands)

_lock = threading.Lock()
_lib = None


class LrqError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__("%s failed with status %d: %s" % (where, status, message))
        self.status = status


LRQ_MATRIX_DENSE_C128 = 0
LRQ_MATRIX_CSR_LAPLACIAN = 1


class LrqMatrix(ctypes.Structure):
    """lrq_matrix of include/lrq.h (array members are device pointers)."""
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int64), ("values", ctypes.c_void_p), ("ld", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("nnz", ctypes.c_int64)]


def dense_matrix(Q: torch.Tensor) -> LrqMatrix:
    assert Q.dtype == torch.complex128 and Q.dim() == 2 and Q.shape[0] == Q.shape[1] and Q.stride(1) == 1
    return LrqMatrix(LRQ_MATRIX_DENSE_C128, Q.shape[0], _addr(Q), Q.stride(0), None, None, None, 0)


def laplacian_matrix(rowptr: torch.Tensor, colidx: torch.Tensor, weights=None) -> LrqMatrix:
    assert rowptr.dtype == torch.int32 and colidx.dtype == torch.int32
    assert weights is None or weights.dtype == torch.float64
    return LrqMatrix(LRQ_MATRIX_CSR_LAPLACIAN, rowptr.numel() - 1, None, 0, _addr(rowptr), _addr(colidx),
                     _addr(weights), colidx.numel())


def _addr(t):
    p = _ptr(t)
    return None if p is None else p.value


class LrqProblem(ctypes.Structure):
    """lrq_problem of include/lrq.h (V and C are device pointers)."""
    _fields_ = [("V", ctypes.c_void_p), ("n", ctypes.c_int64), ("r", ctypes.c_int), ("K", ctypes.c_int),
                ("C", ctypes.c_void_p), ("S", ctypes.c_int64), ("seed", ctypes.c_uint64)]


def load() -> ctypes.CDLL:
    """Load liblrq.so from the package directory (built by build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblrq.so is not built (expected at %s); run __graft_entry__.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        P, I, I64, U64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
        lib.lrq_status_string.argtypes = [I]
        lib.lrq_status_string.restype = ctypes.c_char_p
        lib.lrq_last_error.argtypes = []
        lib.lrq_last_error.restype = ctypes.c_char_p
        lib.lrq_abi_version.argtypes = []
        lib.lrq_abi_version.restype = I
        lib.lrq_sample_directions.argtypes = [U64, I64, I, P, P]
        lib.lrq_sample_directions.restype = I
        lib.lrq_sample_score_workspace_size.argtypes = [I64, I, I, I64, I, I, ctypes.POINTER(SZ)]
        lib.lrq_sample_score_workspace_size.restype = I
        lib.lrq_sample_score.argtypes = [P, I64, I, I, P, I, U64, I64, I, I, P, P, P, P, SZ, P, P]
        lib.lrq_sample_score.restype = I
        lib.lrq_prepared_create.argtypes = [I64, I, I, I, ctypes.POINTER(P)]
        lib.lrq_prepared_create.restype = I
        lib.lrq_prepared_destroy.argtypes = [P]
        lib.lrq_prepared_destroy.restype = None
        lib.lrq_prepared_size.argtypes = [P, ctypes.POINTER(SZ)]
        lib.lrq_prepared_size.restype = I
        lib.lrq_prepare.argtypes = [P, P, P, SZ, P, P]
        lib.lrq_prepare.restype = I
        lib.lrq_sample_score_prepared_workspace_size.argtypes = [P, I64, I, ctypes.POINTER(SZ)]
        lib.lrq_sample_score_prepared_workspace_size.restype = I
        lib.lrq_sample_score_prepared.argtypes = [P, P, I, U64, I64, I, P, P, P, P, SZ, P, P]
        lib.lrq_sample_score_prepared.restype = I
        lib.lrq_rescore_workspace_size.argtypes = [I64, I, I, ctypes.POINTER(SZ)]
        lib.lrq_rescore_workspace_size.restype = I
        lib.lrq_rescore.argtypes = [P, I64, I, I, P, I64, P, I, P, P, P, P, P, SZ, P, P]
        lib.lrq_rescore.restype = I
        lib.lrq_rescore_no_alloc.argtypes = [P, I64, I, I, P, I64, P, I, P, P, P, P, P, P]
        lib.lrq_rescore_no_alloc.restype = I
        PP = ctypes.c_void_p
        lib.lrq_batched_plan_create.argtypes = [ctypes.POINTER(LrqProblem), I, I, ctypes.POINTER(PP)]
        lib.lrq_batched_plan_create.restype = I
        lib.lrq_batched_plan_destroy.argtypes = [PP]
        lib.lrq_batched_plan_destroy.restype = None
        lib.lrq_batched_workspace_size.argtypes = [PP, ctypes.POINTER(SZ)]
        lib.lrq_batched_workspace_size.restype = I
        lib.lrq_batched_prepare.argtypes = [PP, P, SZ, P]
        lib.lrq_batched_prepare.restype = I
        lib.lrq_batched_autotune.argtypes = [PP, P, SZ, P, P]
        lib.lrq_batched_autotune.restype = I
        lib.lrq_batched_tile.argtypes = [PP, I]
        lib.lrq_batched_tile.restype = I
        lib.lrq_sample_score_batched.argtypes = [PP, P, SZ, P, P, P, P]
        lib.lrq_sample_score_batched.restype = I
        lib.lrq_batched_graph_create.argtypes = [PP, P, SZ, P, P, P, P, ctypes.POINTER(PP)]
        lib.lrq_batched_graph_create.restype = I
        lib.lrq_graph_launch.argtypes = [PP, P]
        lib.lrq_graph_launch.restype = I
        lib.lrq_graph_destroy.argtypes = [PP]
        lib.lrq_graph_destroy.restype = I
        F32 = ctypes.c_float
        lib.lrq_proposal_num_features.argtypes = [I]
        lib.lrq_proposal_num_features.restype = I
        lib.lrq_proposal_num_params.argtypes = [I]
        lib.lrq_proposal_num_params.restype = I64
        lib.lrq_proposal_features.argtypes = [P, I, I64, I, P, P, P, P, P]
        lib.lrq_proposal_features.restype = I
        lib.lrq_mlp_forward.argtypes = [P, I, I, P, P, P, P, I, P]
        lib.lrq_mlp_forward.restype = I
        lib.lrq_mlp_backward.argtypes = [P, I, I, P, P, P, P, P, P, I, P]
        lib.lrq_mlp_backward.restype = I
        lib.lrq_vmf_nll.argtypes = [P, I, P, I, P, P, P]
        lib.lrq_vmf_nll.restype = I
        lib.lrq_vmf_sample.argtypes = [P, I, I, I, U64, P, P, P]
        lib.lrq_vmf_sample.restype = I
        lib.lrq_vmf_modes.argtypes = [P, I, P, P]
        lib.lrq_vmf_modes.restype = I
        lib.lrq_adam_step.argtypes = [P, P, P, P, I64, I, F32, F32, F32, F32, P]
        lib.lrq_adam_step.restype = I
        lib.lrq_proposal_targets.argtypes = [P, I64, I, I, P, I64, P, P, P]
        lib.lrq_proposal_targets.restype = I
        lib.lrq_standardize_fit.argtypes = [P, I, I, P, P, P]
        lib.lrq_standardize_fit.restype = I
        lib.lrq_standardize.argtypes = [P, I, I, P, P, P, P]
        lib.lrq_standardize.restype = I
        lib.lrq_truncate_workspace_size.argtypes = [ctypes.POINTER(LrqMatrix), I, I, ctypes.POINTER(SZ)]
        lib.lrq_truncate_workspace_size.restype = I
        lib.lrq_truncate.argtypes = [ctypes.POINTER(LrqMatrix), I, ctypes.c_double, I, U64, P, P, P,
                                     ctypes.POINTER(I64), P, SZ, P, P]
        lib.lrq_truncate.restype = I
        lib.lrq_rank1_workspace_size.argtypes = [I64, ctypes.POINTER(SZ)]
        lib.lrq_rank1_workspace_size.restype = I
        lib.lrq_rank1_sweep.argtypes = [P, I64, I, P, P, P, P, I64, P, P, P, SZ, P, P]
        lib.lrq_rank1_sweep.restype = I
        lib.lrq_sample_null_directions.argtypes = [P, I64, I, I, U64, I64, P, P, P, P]
        lib.lrq_sample_null_directions.restype = I
        lib.lrq_spectral_energy.argtypes = [ctypes.POINTER(LrqMatrix), P, I, P, P, P, P]
        lib.lrq_spectral_energy.restype = I
        lib.lrq_two_eigvec_q.argtypes = [P, I64, I, P, P, P]
        lib.lrq_two_eigvec_q.restype = I
        lib.lrq_greedy_workspace_size.argtypes = [I64, ctypes.POINTER(SZ)]
        lib.lrq_greedy_workspace_size.restype = I
        lib.lrq_greedy_cut.argtypes = [P, P, I64, I64, I, P, I64, P, P, P, P, P, SZ, P, P]
        lib.lrq_greedy_cut.restype = I
        lib.lrq_enumerate_workspace_size.argtypes = [I64, I, I, ctypes.POINTER(SZ)]
        lib.lrq_enumerate_workspace_size.restype = I
        lib.lrq_enumerate.argtypes = [P, I64, I, I, ctypes.c_double, P, P, P, P, SZ, P, P]
        lib.lrq_enumerate.restype = I
        lib.lrq_cut_count.argtypes = [P, P, I64, P, P, P]
        lib.lrq_cut_count.restype = I
        lib.lrq_set_timing_events.argtypes = [P, P]
        lib.lrq_set_timing_events.restype = I
        lib.lrq_kernel_launches.argtypes = []
        lib.lrq_kernel_launches.restype = ctypes.c_uint64
        _lib = lib
        return lib


def exported_symbols():
    """Names of the entry points include/lrq.h declares."""
    return ["lrq_status_string", "lrq_last_error", "lrq_abi_version", "lrq_sample_directions",
            "lrq_sample_score_workspace_size", "lrq_sample_score", "lrq_prepared_create", "lrq_prepared_destroy",
            "lrq_prepared_size", "lrq_prepare", "lrq_sample_score_prepared_workspace_size",
            "lrq_sample_score_prepared", "lrq_rescore_workspace_size",
            "lrq_rescore", "lrq_rescore_no_alloc", "lrq_truncate_workspace_size", "lrq_truncate",
            "lrq_sample_null_directions", "lrq_spectral_energy", "lrq_rank1_workspace_size", "lrq_rank1_sweep", "lrq_two_eigvec_q", "lrq_greedy_workspace_size", "lrq_greedy_cut",
            "lrq_enumerate_workspace_size", "lrq_enumerate", "lrq_batched_plan_create", "lrq_batched_plan_destroy",
            "lrq_batched_workspace_size", "lrq_batched_prepare", "lrq_batched_autotune", "lrq_batched_tile",
            "lrq_sample_score_batched", "lrq_batched_graph_create", "lrq_graph_launch", "lrq_graph_destroy",
            "lrq_proposal_num_features", "lrq_proposal_num_params", "lrq_proposal_features", "lrq_mlp_forward",
            "lrq_mlp_backward", "lrq_vmf_nll", "lrq_vmf_sample", "lrq_vmf_modes", "lrq_adam_step",
            "lrq_proposal_targets", "lrq_standardize_fit", "lrq_standardize",
            "lrq_cut_count", "lrq_set_timing_events", "lrq_kernel_launches"]


def _check(status: int, where: str):
    if status != LRQ_OK:
        lib = load()
        raise LrqError(status, where, lib.lrq_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def lrq_status_string(status: int) -> str:
    return load().lrq_status_string(int(status)).decode()


def lrq_last_error() -> str:
    return load().lrq_last_error().decode()


def lrq_abi_version() -> int:
    return int(load().lrq_abi_version())


def lrq_sample_directions(seed: int, S: int, r: int, C_out: torch.Tensor, stream=None):
    assert C_out.dtype == torch.complex64 and C_out.numel() >= S * r
    _check(load().lrq_sample_directions(int(seed), int(S), int(r), _ptr(C_out), _stream(stream)),
           "lrq_sample_directions")


def lrq_sample_score_workspace_size(n: int, r: int, K: int, S: int, mode: int, top_m: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().lrq_sample_score_workspace_size(int(n), int(r), int(K), int(S), int(mode), int(top_m),
                                                  ctypes.byref(out)), "lrq_sample_score_workspace_size")
    return int(out.value)


def lrq_sample_score(V: torch.Tensor, K: int, C: torch.Tensor, generate_C: bool, seed: int, mode: int,
                     top_m: int, scores_out, top_idx_out: torch.Tensor, top_f_out: torch.Tensor,
                     ws: torch.Tensor, dev_status: torch.Tensor, stream=None):
    n, r = V.shape
    S = C.shape[0]
    assert V.dtype == torch.complex64 and C.dtype == torch.complex64 and C.shape[1] == r
    assert top_idx_out.dtype == torch.int64 and top_f_out.dtype == torch.float32
    assert dev_status.dtype == torch.int32
    _check(load().lrq_sample_score(_ptr(V), n, r, int(K), _ptr(C), int(bool(generate_C)), int(seed), S,
                                   int(mode), int(top_m), _ptr(scores_out), _ptr(top_idx_out), _ptr(top_f_out),
                                   _ptr(ws), ws.numel() * ws.element_size(), _ptr(dev_status), _stream(stream)),
           "lrq_sample_score")


def lrq_rescore_workspace_size(n: int, r: int, m: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().lrq_rescore_workspace_size(int(n), int(r), int(m), ctypes.byref(out)),
           "lrq_rescore_workspace_size")
    return int(out.value)


def lrq_rescore(V: torch.Tensor, K: int, C: torch.Tensor, idx: torch.Tensor, f_out: torch.Tensor, z_out,
                best_out: torch.Tensor, best_f_out: torch.Tensor, ws: torch.Tensor, dev_status: torch.Tensor,
                stream=None):
    n, r = V.shape
    S = C.shape[0]
    m = idx.numel()
    assert idx.dtype == torch.int64 and f_out.dtype == torch.float64
    _check(load().lrq_rescore(_ptr(V), n, r, int(K), _ptr(C), S, _ptr(idx), m, _ptr(f_out), _ptr(z_out),
                              _ptr(best_out), _ptr(best_f_out), _ptr(ws), ws.numel() * ws.element_size(),
                              _ptr(dev_status), _stream(stream)), "lrq_rescore")


def lrq_rescore_no_alloc(V: torch.Tensor, K: int, C: torch.Tensor, idx: torch.Tensor, f_out: torch.Tensor,
                         z_out, best_out: torch.Tensor, best_f_out: torch.Tensor, dev_status: torch.Tensor,
                         stream=None):
    """lrq_rescore for callers that cannot allocate device memory: the library
    uses its own fixed 4 MiB scratch array instead of a workspace."""
    n, r = V.shape
    S = C.shape[0]
    m = idx.numel()
    assert idx.dtype == torch.int64 and f_out.dtype == torch.float64
    _check(load().lrq_rescore_no_alloc(_ptr(V), n, r, int(K), _ptr(C), S, _ptr(idx), m, _ptr(f_out), _ptr(z_out),
                                       _ptr(best_out), _ptr(best_f_out), _ptr(dev_status), _stream(stream)),
           "lrq_rescore_no_alloc")


def lrq_proposal_num_features(r: int) -> int:
    return int(load().lrq_proposal_num_features(int(r)))


def lrq_proposal_num_params(F: int) -> int:
    return int(load().lrq_proposal_num_params(int(F)))


def lrq_proposal_features(V, lam, Vg_out, feat_out, dev_status, stream=None):
    """V: B x n x r complex64; lam: B x r float64; Vg_out like V; feat_out: B x F float32."""
    B, n, r = V.shape
    _check(load().lrq_proposal_features(_ptr(V), B, n, r, _ptr(lam), _ptr(Vg_out), _ptr(feat_out),
                                        _ptr(dev_status), _stream(stream)), "lrq_proposal_features")


def lrq_mlp_forward(params, X, H1, H2, O, bf16=False, stream=None):
    B, F = X.shape
    _check(load().lrq_mlp_forward(_ptr(params), F, B, _ptr(X), _ptr(H1), _ptr(H2), _ptr(O), int(bool(bf16)),
                                  _stream(stream)), "lrq_mlp_forward")


def lrq_mlp_backward(params, X, H1, H2, dO, grads, scratch, bf16=False, stream=None):
    B, F = X.shape
    _check(load().lrq_mlp_backward(_ptr(params), F, B, _ptr(X), _ptr(H1), _ptr(H2), _ptr(dO), _ptr(grads),
                                   _ptr(scratch), int(bool(bf16)), _stream(stream)), "lrq_mlp_backward")


def lrq_vmf_nll(O, targets, loss_out, dO, stream=None):
    B, T, _ = targets.shape
    _check(load().lrq_vmf_nll(_ptr(O), B, _ptr(targets), T, _ptr(loss_out), _ptr(dO), _stream(stream)),
           "lrq_vmf_nll")


def lrq_vmf_sample(O, S, K, seed, C_out, dev_status, stream=None):
    B = O.shape[0]
    _check(load().lrq_vmf_sample(_ptr(O), B, int(S), int(K), int(seed), _ptr(C_out), _ptr(dev_status),
                                 _stream(stream)), "lrq_vmf_sample")


def lrq_vmf_modes(O, C_out, stream=None):
    B = O.shape[0]
    assert O.dtype == torch.float32 and C_out.dtype == torch.complex64 and C_out.numel() == B * 16 * 4
    _check(load().lrq_vmf_modes(_ptr(O), B, _ptr(C_out), _stream(stream)), "lrq_vmf_modes")


def lrq_adam_step(params, grads, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().lrq_adam_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), params.numel(), int(t), float(lr),
                                float(beta1), float(beta2), float(eps), _stream(stream)), "lrq_adam_step")


def lrq_proposal_targets(C, K, idx, targets_out, dev_status, stream=None):
    """C: S x r complex64; idx: m int64; targets_out: m x 2r float32 (device)."""
    S, r = C.shape
    m = idx.numel()
    assert idx.dtype == torch.int64 and targets_out.dtype == torch.float32 and targets_out.numel() == m * 2 * r
    _check(load().lrq_proposal_targets(_ptr(C), S, r, int(K), _ptr(idx), m, _ptr(targets_out), _ptr(dev_status),
                                       _stream(stream)), "lrq_proposal_targets")


def lrq_standardize_fit(feat, mean_out, std_out, stream=None):
    B, F = feat.shape
    _check(load().lrq_standardize_fit(_ptr(feat), B, F, _ptr(mean_out), _ptr(std_out), _stream(stream)),
           "lrq_standardize_fit")


def lrq_standardize(feat, mean, std, X_out, stream=None):
    B, F = feat.shape
    _check(load().lrq_standardize(_ptr(feat), B, F, _ptr(mean), _ptr(std), _ptr(X_out), _stream(stream)),
           "lrq_standardize")


def lrq_truncate_workspace_size(Q: LrqMatrix, r: int, max_iter: int = 0) -> int:
    out = ctypes.c_size_t(0)
    _check(load().lrq_truncate_workspace_size(ctypes.byref(Q), int(r), int(max_iter), ctypes.byref(out)),
           "lrq_truncate_workspace_size")
    return int(out.value)


def lrq_truncate(Q: LrqMatrix, r: int, tol: float, max_iter: int, seed: int, V_out, V32_out, lambda_out,
                 ws: torch.Tensor, dev_status: torch.Tensor, stream=None) -> int:
    """Returns the total number of Lanczos steps."""
    iters = ctypes.c_int64(0)
    _check(load().lrq_truncate(ctypes.byref(Q), int(r), float(tol), int(max_iter), int(seed), _ptr(V_out),
                               _ptr(V32_out), _ptr(lambda_out), ctypes.byref(iters), _ptr(ws),
                               ws.numel() * ws.element_size(), _ptr(dev_status), _stream(stream)), "lrq_truncate")
    return int(iters.value)


def lrq_rank1_workspace_size(n: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().lrq_rank1_workspace_size(int(n), ctypes.byref(out)), "lrq_rank1_workspace_size")
    return int(out.value)


def lrq_rank1_sweep(q, K, z_out, f_out, rowptr, colidx, cut_out, zcut_out, ws, dev_status, stream=None):
    """q: n complex128 (device); rowptr/colidx: int32 CSR or None."""
    n = q.numel()
    nnz = 0 if colidx is None else colidx.numel()
    _check(load().lrq_rank1_sweep(_ptr(q), n, int(K), _ptr(z_out), _ptr(f_out), _ptr(rowptr), _ptr(colidx), nnz,
                                  _ptr(cut_out), _ptr(zcut_out), _ptr(ws), ws.numel() * ws.element_size(),
                                  _ptr(dev_status), _stream(stream)), "lrq_rank1_sweep")


def lrq_sample_null_directions(V, K, seed, S, C_out, draws_out, dev_status, stream=None):
    """V: n x r complex64 (device); C_out: S x r complex64; draws_out: 1 int64."""
    n, r = V.shape
    _check(load().lrq_sample_null_directions(_ptr(V), n, r, int(K), int(seed), int(S), _ptr(C_out), _ptr(draws_out),
                                             _ptr(dev_status), _stream(stream)), "lrq_sample_null_directions")


def sample_null_directions(V, K, S, seed, stream=None):
    """S null-vector directions (randomised Algorithm 2) and the draw count."""
    C = torch.empty((S, V.shape[1]), dtype=torch.complex64, device=V.device)
    draws = torch.zeros(1, dtype=torch.int64, device=V.device)
    st = torch.zeros(1, dtype=torch.int32, device=V.device)
    lrq_sample_null_directions(V, K, seed, S, C, draws, st, stream)
    return dict(C=C, draws=draws, dev_status=st)


def lrq_spectral_energy(Q, lam, trace_out, rho_out, dev_status, stream=None):
    """Q: LrqMatrix; lam: r float64 (device)."""
    _check(load().lrq_spectral_energy(ctypes.byref(Q), _ptr(lam), lam.numel(), _ptr(trace_out), _ptr(rho_out),
                                      _ptr(dev_status), _stream(stream)), "lrq_spectral_energy")


def spectral_energy(Q, lam, device="cuda", stream=None):
    """rho_r = 1 - sum of the top r eigenvalues / trace(Q), and trace(Q)."""
    tr = torch.zeros(1, dtype=torch.float64, device=device)
    rho = torch.zeros(1, dtype=torch.float64, device=device)
    st = torch.zeros(1, dtype=torch.int32, device=device)
    lrq_spectral_energy(Q, lam, tr, rho, st, stream)
    return dict(rho=rho, trace=tr, dev_status=st)


def lrq_two_eigvec_q(V, lam, q_out, stream=None):
    """V: n x r complex128 (device, r >= 2); lam: r float64 (device)."""
    n, r = V.shape
    _check(load().lrq_two_eigvec_q(_ptr(V), n, r, _ptr(lam), _ptr(q_out), _stream(stream)), "lrq_two_eigvec_q")


def two_eigvec_q(V, lam, stream=None):
    """q = u_1 + i u_2 from a real truncation (two-eigenvector rounding)."""
    q = torch.empty(V.shape[0], dtype=torch.complex128, device=V.device)
    lrq_two_eigvec_q(V, lam, q, stream)
    return q


def lrq_greedy_workspace_size(n: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().lrq_greedy_workspace_size(int(n), ctypes.byref(out)), "lrq_greedy_workspace_size")
    return int(out.value)


def lrq_greedy_cut(rowptr, colidx, K, z, max_rounds, cut_out, ws, dev_status, stream=None):
    """rowptr/colidx: int32 CSR (device); z: n uint8 labels (device), refined
    in place.  Returns (rounds that moved, vertices moved, converged)."""
    n = z.numel()
    nnz = colidx.numel()
    rounds, moves, conv = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int32(0)
    _check(load().lrq_greedy_cut(_ptr(rowptr), _ptr(colidx), n, nnz, int(K), _ptr(z), int(max_rounds),
                                 _ptr(cut_out), ctypes.byref(rounds), ctypes.byref(moves), ctypes.byref(conv),
                                 _ptr(ws), ws.numel() * ws.element_size(), _ptr(dev_status), _stream(stream)),
           "lrq_greedy_cut")
    return int(rounds.value), int(moves.value), bool(conv.value)


def lrq_enumerate_workspace_size(n: int, r: int, K: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().lrq_enumerate_workspace_size(int(n), int(r), int(K), ctypes.byref(out)),
           "lrq_enumerate_workspace_size")
    return int(out.value)


def lrq_enumerate(V: torch.Tensor, K: int, budget: float, z_out: torch.Tensor, f_out: torch.Tensor, n_sets_out,
                  ws: torch.Tensor, dev_status: torch.Tensor, stream=None):
    """V: n x r complex128 on the device."""
    n, r = V.shape
    assert V.dtype == torch.complex128 and z_out.dtype == torch.uint8 and f_out.dtype == torch.float64
    _check(load().lrq_enumerate(_ptr(V), n, r, int(K), float(budget), _ptr(z_out), _ptr(f_out), _ptr(n_sets_out),
                                _ptr(ws), ws.numel() * ws.element_size(), _ptr(dev_status), _stream(stream)),
           "lrq_enumerate")


def lrq_cut_count(rowptr: torch.Tensor, colidx: torch.Tensor, z: torch.Tensor, cut_out: torch.Tensor,
                  stream=None):
    assert rowptr.dtype == torch.int32 and colidx.dtype == torch.int32 and z.dtype == torch.uint8
    _check(load().lrq_cut_count(_ptr(rowptr), _ptr(colidx), rowptr.numel() - 1, _ptr(z), _ptr(cut_out),
                                _stream(stream)), "lrq_cut_count")


def lrq_set_timing_events(start_event, stop_event):
    """start_event / stop_event: torch.cuda.Event(enable_timing=True) or None."""
    for ev in (start_event, stop_event):
        if ev is not None and not ev.cuda_event:
            ev.record()  # torch creates the underlying cudaEvent lazily, on first record
    a = None if start_event is None else ctypes.c_void_p(start_event.cuda_event)
    b = None if stop_event is None else ctypes.c_void_p(stop_event.cuda_event)
    _check(load().lrq_set_timing_events(a, b), "lrq_set_timing_events")


def lrq_kernel_launches() -> int:
    return int(load().lrq_kernel_launches())


# --------------------------------------------------------------------------
# Convenience wrappers (allocate outputs and workspace with torch).
# --------------------------------------------------------------------------
def workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def check_status(dev_status: torch.Tensor, where: str = "device"):
    s = int(dev_status.item())
    if s != LRQ_OK:
        raise LrqError(s, where, lrq_status_string(s))


def sample_score(V, K, C=None, S=None, seed=0, mode=LRQ_MODE_TC, top_m=64, want_scores=False,
                 ws=None, dev_status=None, stream=None):
    """Score S directions (given in C, or drawn from `seed` into a new C).
    Returns dict(C, top_idx, top_f, scores, dev_status)."""
    dev = V.device
    n, r = V.shape
    generate = C is None
    if generate:
        C = torch.empty((int(S), r), dtype=torch.complex64, device=dev)
    S = C.shape[0]
    need = lrq_sample_score_workspace_size(n, r, K, S, mode, top_m)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    if dev_status is None:
        dev_status = torch.zeros(1, dtype=torch.int32, device=dev)
    top_idx = torch.empty(top_m, dtype=torch.int64, device=dev)
    top_f = torch.empty(top_m, dtype=torch.float32, device=dev)
    scores = torch.empty(S, dtype=torch.float32, device=dev) if want_scores else None
    lrq_sample_score(V, K, C, generate, seed, mode, top_m, scores, top_idx, top_f, ws, dev_status, stream)
    return dict(C=C, top_idx=top_idx, top_f=top_f, scores=scores, dev_status=dev_status, ws=ws)


def rescore(V, K, C, idx, want_z=False, ws=None, dev_status=None, stream=None):
    dev = V.device
    n, r = V.shape
    m = idx.numel()
    need = lrq_rescore_workspace_size(n, r, m)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    if dev_status is None:
        dev_status = torch.zeros(1, dtype=torch.int32, device=dev)
    f = torch.empty(m, dtype=torch.float64, device=dev)
    z = torch.empty((m, n), dtype=torch.uint8, device=dev) if want_z else None
    best = torch.empty(1, dtype=torch.int64, device=dev)
    best_f = torch.empty(1, dtype=torch.float64, device=dev)
    lrq_rescore(V, K, C, idx, f, z, best, best_f, ws, dev_status, stream)
    return dict(f=f, z=z, best=best, best_f=best_f, dev_status=dev_status, ws=ws)


def enumerate_exact(V, K, budget=0.0, stream=None):
    """Exact maximiser for rank r; allocates outputs and workspace with torch."""
    dev = V.device
    n, r = V.shape
    ws = workspace(lrq_enumerate_workspace_size(n, r, K), dev)
    dev_status = torch.zeros(1, dtype=torch.int32, device=dev)
    z = torch.empty(n, dtype=torch.uint8, device=dev)
    f = torch.empty(1, dtype=torch.float64, device=dev)
    n_sets = torch.empty(1, dtype=torch.int64, device=dev)
    lrq_enumerate(V, K, budget, z, f, n_sets, ws, dev_status, stream)
    return dict(z=z, f=f, n_sets=n_sets, dev_status=dev_status)


def truncate(Q: LrqMatrix, r, tol=0.0, max_iter=0, seed=0, want_c128=True, want_c64=True, device="cuda",
             stream=None):
    """Top-r spectral truncation; keep the tensors behind Q alive meanwhile."""
    n = Q.n
    ws = workspace(lrq_truncate_workspace_size(Q, r, max_iter), device)
    dev_status = torch.zeros(1, dtype=torch.int32, device=device)
    V = torch.empty((n, r), dtype=torch.complex128, device=device) if want_c128 else None
    V32 = torch.empty((n, r), dtype=torch.complex64, device=device) if want_c64 else None
    lam = torch.empty(r, dtype=torch.float64, device=device)
    iters = lrq_truncate(Q, r, tol, max_iter, seed, V, V32, lam, ws, dev_status, stream)
    return dict(V=V, V32=V32, lam=lam, iters=iters)


class BatchedPlan:
    """Owns an lrq_batched_plan, its workspace and outputs; keeps the problem
    tensors alive.  problems: list of dicts with V (n x r complex64, device),
    K, and either C (S x r complex64, device), or S and seed, or exact=True
    (S = 0: solved exactly by vertex enumeration in the same launch)."""

    def __init__(self, problems, top_m=4, device="cuda", stream=None):
        self.keep = []
        arr = (LrqProblem * len(problems))()
        for i, q in enumerate(problems):
            V = q["V"]
            C = q.get("C")
            self.keep += [V, C]
            S = 0 if q.get("exact") else (C.shape[0] if C is not None else int(q["S"]))
            arr[i] = LrqProblem(_addr(V), V.shape[0], V.shape[1], int(q["K"]), _addr(C), S, int(q.get("seed", 0)))
        h = ctypes.c_void_p()
        _check(load().lrq_batched_plan_create(arr, len(problems), int(top_m), ctypes.byref(h)),
               "lrq_batched_plan_create")
        self.h = h
        self.P = len(problems)
        self.stream = stream
        nb = ctypes.c_size_t(0)
        _check(load().lrq_batched_workspace_size(self.h, ctypes.byref(nb)), "lrq_batched_workspace_size")
        self.ws = workspace(nb.value, device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.best_f = torch.empty(self.P, dtype=torch.float64, device=device)
        self.best_idx = torch.empty(self.P, dtype=torch.int64, device=device)
        self.graph = None
        _check(load().lrq_batched_prepare(self.h, _ptr(self.ws), self._wsb(), _stream(stream)), "lrq_batched_prepare")

    def _wsb(self):
        return self.ws.numel() * self.ws.element_size()

    def autotune(self):
        _check(load().lrq_batched_autotune(self.h, _ptr(self.ws), self._wsb(), _ptr(self.status),
                                           _stream(self.stream)), "lrq_batched_autotune")

    def tile(self, p):
        return int(load().lrq_batched_tile(self.h, int(p)))

    def run(self):
        _check(load().lrq_sample_score_batched(self.h, _ptr(self.ws), self._wsb(), _ptr(self.best_f),
                                               _ptr(self.best_idx), _ptr(self.status), _stream(self.stream)),
               "lrq_sample_score_batched")

    def capture(self):
        g = ctypes.c_void_p()
        _check(load().lrq_batched_graph_create(self.h, _ptr(self.ws), self._wsb(), _ptr(self.best_f),
                                               _ptr(self.best_idx), _ptr(self.status), _stream(self.stream),
                                               ctypes.byref(g)), "lrq_batched_graph_create")
        self.graph = g

    def replay(self):
        _check(load().lrq_graph_launch(self.graph, _stream(self.stream)), "lrq_graph_launch")

    def close(self):
        if self.graph is not None:
            load().lrq_graph_destroy(self.graph)
            self.graph = None
        if self.h:
            load().lrq_batched_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PreparedInstance:
    """Owns an lrq_prepared_v handle and its device buffer; keeps V alive.
    prepare(V) packs V's operands once; sample_score(...) then scores
    directions against them (same results as the module-level sample_score)."""

    def __init__(self, n, r, K, mode=LRQ_MODE_TC, device="cuda"):
        h = ctypes.c_void_p()
        _check(load().lrq_prepared_create(int(n), int(r), int(K), int(mode), ctypes.byref(h)), "lrq_prepared_create")
        self.h = h
        self.n, self.r, self.K, self.mode, self.device = int(n), int(r), int(K), int(mode), device
        nb = ctypes.c_size_t(0)
        _check(load().lrq_prepared_size(self.h, ctypes.byref(nb)), "lrq_prepared_size")
        self.nbytes = int(nb.value)
        self.buf = workspace(self.nbytes, device) if self.nbytes else None
        self.V = None
        self.dev_status = torch.zeros(1, dtype=torch.int32, device=device)

    def prepare(self, V, stream=None):
        assert V.dtype == torch.complex64 and tuple(V.shape) == (self.n, self.r)
        bb = self.buf.numel() if self.buf is not None else 0
        _check(load().lrq_prepare(self.h, _ptr(V), _ptr(self.buf), bb, _ptr(self.dev_status), _stream(stream)),
               "lrq_prepare")
        self.V = V
        return self

    def workspace_size(self, S, top_m):
        out = ctypes.c_size_t(0)
        _check(load().lrq_sample_score_prepared_workspace_size(self.h, int(S), int(top_m), ctypes.byref(out)),
               "lrq_sample_score_prepared_workspace_size")
        return int(out.value)

    def score_into(self, C, generate_C, seed, top_m, scores_out, top_idx_out, top_f_out, ws, dev_status,
                   stream=None):
        assert C.dtype == torch.complex64 and C.shape[1] == self.r
        _check(load().lrq_sample_score_prepared(self.h, _ptr(C), int(bool(generate_C)), int(seed), C.shape[0],
                                                int(top_m), _ptr(scores_out), _ptr(top_idx_out), _ptr(top_f_out),
                                                _ptr(ws), ws.numel() * ws.element_size(), _ptr(dev_status),
                                                _stream(stream)), "lrq_sample_score_prepared")

    def sample_score(self, C=None, S=None, seed=0, top_m=64, want_scores=False, ws=None, dev_status=None,
                     stream=None):
        dev = self.device
        generate = C is None
        if generate:
            C = torch.empty((int(S), self.r), dtype=torch.complex64, device=dev)
        S = C.shape[0]
        need = self.workspace_size(S, top_m)
        if ws is None or ws.numel() < need:
            ws = workspace(need, dev)
        if dev_status is None:
            dev_status = torch.zeros(1, dtype=torch.int32, device=dev)
        top_idx = torch.empty(top_m, dtype=torch.int64, device=dev)
        top_f = torch.empty(top_m, dtype=torch.float32, device=dev)
        scores = torch.empty(S, dtype=torch.float32, device=dev) if want_scores else None
        self.score_into(C, generate, seed, top_m, scores, top_idx, top_f, ws, dev_status, stream)
        return dict(C=C, top_idx=top_idx, top_f=top_f, scores=scores, dev_status=dev_status, ws=ws)

    def close(self):
        if self.h:
            load().lrq_prepared_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rank1_sweep(q, K, rowptr=None, colidx=None, stream=None):
    """Exact rank-1 optimum (and, with a graph, the best-cut state of the sweep)."""
    dev = q.device
    n = q.numel()
    ws = workspace(lrq_rank1_workspace_size(n), dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    z = torch.empty(n, dtype=torch.uint8, device=dev)
    f = torch.empty(1, dtype=torch.float64, device=dev)
    cut = torch.zeros(1, dtype=torch.int64, device=dev) if rowptr is not None else None
    zc = torch.empty(n, dtype=torch.uint8, device=dev) if rowptr is not None else None
    lrq_rank1_sweep(q, K, z, f, rowptr, colidx, cut, zc, ws, st, stream)
    return dict(z=z, f=f, cut=cut, zcut=zc, dev_status=st)


def greedy_cut(rowptr, colidx, K, z, max_rounds=1 << 20, stream=None):
    """Greedy Max-K-Cut local search from the labels z (left untouched; the
    refined labels are returned): the hybrid solver's second step when z is
    the rank-1 sweep's best-cut state."""
    dev = z.device
    zz = z.clone()
    ws = workspace(lrq_greedy_workspace_size(zz.numel()), dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    cut = torch.zeros(1, dtype=torch.int64, device=dev)
    rounds, moves, conv = lrq_greedy_cut(rowptr, colidx, K, zz, max_rounds, cut, ws, st, stream)
    return dict(z=zz, cut=cut, rounds=rounds, moves=moves, converged=conv, dev_status=st)
