"""Thin Python binding of librsvd.so, the GB300 randomized-SVD library.

Every function here marshals arguments (torch tensors -> device pointers, the
current CUDA stream) and calls the C ABI declared in include/rsvd.h, under the
same name.  All arithmetic happens in the library's CUDA kernels; there is no
CPU or PyTorch fallback: if the library is missing, importing this package
fails loudly.

Convenience wrappers (``fixed_rank``, ``adaptive_tol``, ``orth``, ``sketch``)
allocate outputs and workspace with torch and then make the same C calls.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librsvd.so")

RSVD_OK = 0
RSVD_E_INVALID = 1
RSVD_E_NOMEM = 2
RSVD_E_CUDA = 3
RSVD_E_BREAKDOWN = 4
RSVD_E_NOT_CONVERGED = 5
RSVD_E_NONFINITE = 6
RSVD_E_TIMEOUT = 7
RSVD_E_UNSUPPORTED = 8

RSVD_F64 = 0
RSVD_F32 = 1
RSVD_MIXED_BF16 = 2
RSVD_MIXED_FP8 = 3
RSVD_MIXED_FP8_B128 = 4

RSVD_DT_F64 = 0
RSVD_DT_F32 = 1
RSVD_DT_BF16 = 2

RSVD_FLAG_RETURN_FULL_L = 1
RSVD_FLAG_SYNC = 2
RSVD_FLAG_CERTIFY = 4
RSVD_FLAG_USE_CONTROLLER = 8
RSVD_FLAG_SPECTRAL = 16
RSVD_FLAG_CENTER = 32
RSVD_FLAG_KRYLOV = 64
RSVD_FLAG_SINGLE_PASS = 128
RSVD_FLAG_SYMMETRIC = 256
RSVD_FLAG_SRFT = 512

STATUS_NAMES = {0: "RSVD_OK", 1: "RSVD_E_INVALID", 2: "RSVD_E_NOMEM", 3: "RSVD_E_CUDA", 4: "RSVD_E_BREAKDOWN",
                5: "RSVD_E_NOT_CONVERGED", 6: "RSVD_E_NONFINITE", 7: "RSVD_E_TIMEOUT", 8: "RSVD_E_UNSUPPORTED"}

# Every symbol include/rsvd.h declares (checked by the CPU test suite).
EXPORTED = [
    "rsvd_create", "rsvd_destroy", "rsvd_workspace_size", "rsvd_fixed_rank", "rsvd_adaptive_tol",
    "rsvd_query_status", "rsvd_last_error_detail", "rsvd_philox_words", "rsvd_gaussian",
    "rsvd_sketch_workspace_size", "rsvd_sketch", "rsvd_orth_workspace_size", "rsvd_orth",
    "rsvd_project_workspace_size", "rsvd_project", "rsvd_kernel_launches", "rsvd_profile", "rsvd_profile_read",
    "rsvd_sketch_noalloc", "rsvd_batched_workspace_size", "rsvd_batched",
    "rsvd_probe_workspace_size", "rsvd_probe_features", "rsvd_mlp_workspace_size", "rsvd_mlp_forward",
    "rsvd_mlp_grad", "rsvd_mlp_train_step", "rsvd_controller_attach", "rsvd_controller_last",
    "rsvd_controller_fallback", "rsvd_batched_variants", "rsvd_batched_variant_info", "rsvd_batched_set_variant",
    "rsvd_batched_get_variant", "rsvd_batched_autotune", "rsvd_certify_workspace_size", "rsvd_certify",
    "rsvd_nystrom",
]

CTRL_D_IN = 17
CTRL_HIDDEN = 128
CTRL_OUT = 20
CTRL_PARAMS = 21396


class Params(ctypes.Structure):
    """Mirror of rsvd_params."""
    _fields_ = [("k", ctypes.c_int), ("p", ctypes.c_int), ("q", ctypes.c_int), ("block", ctypes.c_int),
                ("max_rank", ctypes.c_int), ("probe_cols", ctypes.c_int), ("tol", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("prec", ctypes.c_int), ("flags", ctypes.c_int)]


class RsvdError(RuntimeError):
    def __init__(self, code, detail=""):
        self.code = code
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, str(code)), detail))


_lib = None


def load():
    """Load librsvd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("librsvd.so not found at %s; build it with `python -m paper_1607_01649_gb300.build`"
                          % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, u32, u64, sz, dp = (ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                               ctypes.c_size_t, ctypes.c_void_p)
    P = ctypes.POINTER(Params)
    sig = {
        "rsvd_create": [ctypes.POINTER(vp), i],
        "rsvd_destroy": [vp],
        "rsvd_workspace_size": [vp, i, i, P, ctypes.POINTER(sz)],
        "rsvd_fixed_rank": [vp, i, i, vp, i, P, vp, i, dp, vp, i, vp, sz, vp],
        "rsvd_adaptive_tol": [vp, i, i, vp, i, P, vp, i, dp, vp, i, vp, vp, vp, sz, vp],
        "rsvd_query_status": [vp, vp, ctypes.POINTER(i), vp],
        "rsvd_last_error_detail": [vp, ctypes.c_char_p, sz],
        "rsvd_philox_words": [vp, i, i, u64, u32, i, vp, vp],
        "rsvd_gaussian": [vp, i, i, u64, u32, i, i, vp, i, vp],
        "rsvd_sketch_workspace_size": [vp, i, i, i, i, i, ctypes.POINTER(sz)],
        "rsvd_sketch": [vp, i, i, i, i, i, vp, i, vp, i, vp, i, vp, sz, vp],
        "rsvd_orth_workspace_size": [vp, i, i, i, ctypes.POINTER(sz)],
        "rsvd_orth": [vp, i, i, i, vp, i, dp, vp, sz, vp],
        "rsvd_project_workspace_size": [vp, i, i, i, i, ctypes.POINTER(sz)],
        "rsvd_project": [vp, i, i, i, i, vp, i, vp, i, vp, i, vp, sz, vp],
        "rsvd_kernel_launches": [vp, ctypes.POINTER(ctypes.c_longlong)],
        "rsvd_profile": [vp, i],
        "rsvd_profile_read": [vp, i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)],
        "rsvd_sketch_noalloc": [vp, i, i, i, i, vp, i, vp, i, vp, i, vp, vp],
        "rsvd_batched_workspace_size": [vp, i, P, ctypes.POINTER(sz)],
        "rsvd_batched": [vp, i, vp, vp, vp, vp, P, vp, vp, vp, vp, vp, vp, vp, sz, vp],
        "rsvd_batched_variants": [ctypes.POINTER(i)],
        "rsvd_batched_variant_info": [i, ctypes.POINTER(i), ctypes.POINTER(i)],
        "rsvd_batched_set_variant": [vp, i],
        "rsvd_batched_get_variant": [vp, ctypes.POINTER(i)],
        "rsvd_batched_autotune": [vp, i, vp, vp, vp, vp, P, vp, vp, vp, vp, vp, vp, vp, sz, vp, vp, vp],
        "rsvd_certify_workspace_size": [vp, i, i, i, ctypes.POINTER(sz)],
        "rsvd_nystrom": [vp, i, vp, i, P, vp, i, dp, vp, sz, vp],
        "rsvd_certify": [vp, i, i, vp, i, i, vp, i, vp, vp, i, u64, vp, vp, sz, vp],
        "rsvd_probe_workspace_size": [vp, i, i, ctypes.POINTER(sz)],
        "rsvd_probe_features": [vp, i, i, vp, i, u64, vp, vp, vp, sz, vp],
        "rsvd_mlp_workspace_size": [vp, i, ctypes.POINTER(sz)],
        "rsvd_mlp_forward": [vp, i, vp, vp, vp, vp],
        "rsvd_mlp_grad": [vp, i, vp, vp, vp, ctypes.c_float, vp, vp, vp, vp, sz, vp],
        "rsvd_mlp_train_step": [vp, i, vp, vp, vp, ctypes.c_float, vp, vp, vp, i, ctypes.c_float, vp, vp, sz, vp],
        "rsvd_controller_attach": [vp, vp, ctypes.c_double, ctypes.c_double],
        "rsvd_controller_last": [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)],
        "rsvd_controller_fallback": [vp, i],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    _lib = lib
    return lib


_handles = {}


def handle(device=None):
    """A library handle for `device` (cached per device)."""
    import torch
    if device is None:
        device = torch.cuda.current_device()
    if device not in _handles:
        h = ctypes.c_void_p()
        _check(load().rsvd_create(ctypes.byref(h), int(device)), None)
        _handles[device] = h
    return _handles[device]


def last_error(h):
    buf = ctypes.create_string_buffer(512)
    load().rsvd_last_error_detail(h, buf, 512)
    return buf.value.decode(errors="replace")


def _check(code, h):
    if code != RSVD_OK:
        raise RsvdError(code, last_error(h) if h is not None else "")
    return code


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _empty_ws(nbytes, device):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# ---------------------------------------------------------------- raw calls --
def rsvd_workspace_size(h, m, n, params):
    out = ctypes.c_size_t()
    _check(load().rsvd_workspace_size(h, m, n, ctypes.byref(params), ctypes.byref(out)), h)
    return out.value


def rsvd_fixed_rank(h, m, n, A, lda, params, U, ldu, D, V, ldv, ws, stream=None):
    return load().rsvd_fixed_rank(h, m, n, _ptr(A), lda, ctypes.byref(params), _ptr(U), ldu, _ptr(D), _ptr(V), ldv,
                                  _ptr(ws), ws.numel() if ws is not None else 0, _stream(stream))


def rsvd_adaptive_tol(h, m, n, A, lda, params, U, ldu, D, V, ldv, rank_out, err_out, ws, stream=None):
    return load().rsvd_adaptive_tol(h, m, n, _ptr(A), lda, ctypes.byref(params), _ptr(U), ldu, _ptr(D), _ptr(V),
                                    ldv, _ptr(rank_out), _ptr(err_out), _ptr(ws),
                                    ws.numel() if ws is not None else 0, _stream(stream))


def rsvd_batched_workspace_size(h, count, params):
    out = ctypes.c_size_t()
    _check(load().rsvd_batched_workspace_size(h, count, ctypes.byref(params), ctypes.byref(out)), h)
    return out.value


def rsvd_batched(h, count, m, n, A, lda, params, U, D, V, rank_out, err_out, status_out, ws, stream=None):
    return load().rsvd_batched(h, count, _ptr(m), _ptr(n), _ptr(A), _ptr(lda), ctypes.byref(params), _ptr(U),
                               _ptr(D), _ptr(V), _ptr(rank_out), _ptr(err_out), _ptr(status_out), _ptr(ws),
                               ws.numel() if ws is not None else 0, _stream(stream))


def rsvd_batched_variants():
    out = ctypes.c_int()
    _check(load().rsvd_batched_variants(ctypes.byref(out)), None)
    return out.value


def rsvd_batched_variant_info(v):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().rsvd_batched_variant_info(int(v), ctypes.byref(a), ctypes.byref(b)), None)
    return a.value, b.value


def rsvd_batched_set_variant(h, v):
    return _check(load().rsvd_batched_set_variant(h, int(v)), h)


def rsvd_batched_get_variant(h):
    out = ctypes.c_int()
    _check(load().rsvd_batched_get_variant(h, ctypes.byref(out)), h)
    return out.value


def rsvd_batched_autotune(h, count, m, n, A, lda, params, U, D, V, rank_out, err_out, status_out, ws, stream=None):
    """Returns (status, chosen variant, list of per-variant ms)."""
    nv = rsvd_batched_variants()
    ms = (ctypes.c_float * nv)()
    var = ctypes.c_int(-1)
    code = load().rsvd_batched_autotune(h, count, _ptr(m), _ptr(n), _ptr(A), _ptr(lda), ctypes.byref(params),
                                        _ptr(U), _ptr(D), _ptr(V), _ptr(rank_out), _ptr(err_out), _ptr(status_out),
                                        _ptr(ws), ws.numel() if ws is not None else 0, _stream(stream), ms,
                                        ctypes.byref(var))
    return code, var.value, list(ms)


def rsvd_nystrom(h, n, A, lda, params, U, ldu, Lam, ws, stream=None):
    return load().rsvd_nystrom(h, n, _ptr(A), lda, ctypes.byref(params), _ptr(U), ldu, _ptr(Lam), _ptr(ws),
                               ws.numel() if ws is not None else 0, _stream(stream))


def nystrom(A, k, p=10, seed=0, prec=RSVD_F32, full=False, sync=True):
    """A ~= U diag(Lam) U^T by rsvd_nystrom (Fig. nystrom) for a symmetric
    positive semi-definite CUDA tensor A (float64 for RSVD_F64, else
    float32).  Returns (U, Lam)."""
    import torch
    h = handle(A.device.index)
    n = A.shape[0]
    flags = (RSVD_FLAG_RETURN_FULL_L if full else 0) | (RSVD_FLAG_SYNC if sync else 0)
    prm = make_params(k, p, 0, seed, prec, flags)
    kk = k + p if full else k
    U = torch.empty(n, kk, dtype=_prec_dtype(prec), device=A.device)
    Lam = torch.empty(kk, dtype=torch.float64, device=A.device)
    ws = _empty_ws(rsvd_workspace_size(h, n, n, prm), A.device)
    _check(rsvd_nystrom(h, n, A, A.stride(0), prm, U, U.stride(0), Lam, ws), h)
    return U, Lam


def certify(A, U, D, V, seed=0, stream=None):
    """rsvd_certify: (Frobenius estimate, spectral bound, ||A||_F) of
    A - U diag(D) V^T from 16 Gaussian columns of Philox stream 2 (Sec. 14).
    A, U, V float32 and D float64, CUDA or pinned host tensors."""
    h = handle(A.device.index if A.is_cuda else 0)
    m, n = A.shape
    r = 0 if U is None else U.shape[1]
    sz = ctypes.c_size_t()
    _check(load().rsvd_certify_workspace_size(h, m, n, r, ctypes.byref(sz)), h)
    ws = _empty_ws(sz.value, A.device if A.is_cuda else "cuda")
    out = (ctypes.c_double * 3)()
    _check(load().rsvd_certify(h, m, n, _ptr(A), A.stride(0), r, _ptr(U), U.stride(0) if r else 1, _ptr(D),
                               _ptr(V), V.stride(0) if r else 1, int(seed), out, _ptr(ws), ws.numel(),
                               _stream(stream)), h)
    return out[0], out[1], out[2]


def rsvd_query_status(h, ws, stream=None):
    st = ctypes.c_int()
    _check(load().rsvd_query_status(h, _ptr(ws), ctypes.byref(st), _stream(stream)), h)
    return st.value


def rsvd_philox_words(h, n_groups, l, seed, stream_id, col0, out, stream=None):
    return load().rsvd_philox_words(h, n_groups, l, seed, stream_id, col0, _ptr(out), _stream(stream))


def rsvd_gaussian(h, n, l, seed, stream_id, col0, dtype, out, ldo, stream=None):
    return load().rsvd_gaussian(h, n, l, seed, stream_id, col0, dtype, _ptr(out), ldo, _stream(stream))


def rsvd_sketch_workspace_size(h, prec, trans, m, n, l):
    out = ctypes.c_size_t()
    _check(load().rsvd_sketch_workspace_size(h, prec, trans, m, n, l, ctypes.byref(out)), h)
    return out.value


def rsvd_sketch(h, prec, trans, m, n, l, A, lda, X, ldx, Y, ldy, ws, stream=None):
    return load().rsvd_sketch(h, prec, trans, m, n, l, _ptr(A), lda, _ptr(X), ldx, _ptr(Y), ldy, _ptr(ws),
                              ws.numel() if ws is not None else 0, _stream(stream))


def rsvd_orth_workspace_size(h, prec, rows, l):
    out = ctypes.c_size_t()
    _check(load().rsvd_orth_workspace_size(h, prec, rows, l, ctypes.byref(out)), h)
    return out.value


def rsvd_orth(h, prec, rows, l, Y, ldy, R, ws, stream=None):
    return load().rsvd_orth(h, prec, rows, l, _ptr(Y), ldy, _ptr(R), _ptr(ws), ws.numel() if ws is not None else 0,
                            _stream(stream))


def status_block(ws):
    """Diagnostic fields of the device status block at the start of a workspace:
    code, CholeskyQR shift flag, Jacobi sweeps of the last small SVD, number
    of shifted Cholesky factorizations."""
    import numpy as np
    raw = ws[:32].cpu().numpy().view(np.int32)
    return {"code": int(raw[0]), "shifted": int(raw[1]), "jacobi_sweeps": int(raw[3]), "shift_count": int(raw[6])}


def rsvd_project_workspace_size(h, prec, m, n, l):
    out = ctypes.c_size_t()
    _check(load().rsvd_project_workspace_size(h, prec, m, n, l, ctypes.byref(out)), h)
    return out.value


def rsvd_project(h, prec, m, n, l, A, lda, Q, ldq, Bt, ldb, ws, stream=None):
    return load().rsvd_project(h, prec, m, n, l, _ptr(A), lda, _ptr(Q), ldq, _ptr(Bt), ldb, _ptr(ws),
                               ws.numel() if ws is not None else 0, _stream(stream))


def rsvd_sketch_noalloc(h, trans, m, n, l, A, lda, X, ldx, Y, ldy, status=None, stream=None):
    """bf16 tensor-core sketch product with library-owned scratch (no workspace
    argument); `status` (optional) is a one-element int32 device tensor that
    receives the call's device status word."""
    return load().rsvd_sketch_noalloc(h, trans, m, n, l, _ptr(A), lda, _ptr(X), ldx, _ptr(Y), ldy,
                                      _ptr(status) if status is not None else None, _stream(stream))


def rsvd_probe_workspace_size(h, m, n):
    out = ctypes.c_size_t()
    _check(load().rsvd_probe_workspace_size(h, m, n, ctypes.byref(out)), h)
    return out.value


def rsvd_probe_features(h, m, n, A, lda, seed, feat, fro2, ws, stream=None):
    return load().rsvd_probe_features(h, m, n, _ptr(A), lda, seed, _ptr(feat), _ptr(fro2), _ptr(ws),
                                      ws.numel() if ws is not None else 0, _stream(stream))


def rsvd_mlp_workspace_size(h, batch):
    out = ctypes.c_size_t()
    _check(load().rsvd_mlp_workspace_size(h, batch, ctypes.byref(out)), h)
    return out.value


def rsvd_mlp_forward(h, batch, X, theta, logits, stream=None):
    return load().rsvd_mlp_forward(h, batch, _ptr(X), _ptr(theta), _ptr(logits), _stream(stream))


def rsvd_mlp_grad(h, batch, X, yl, yq, lam, theta, grad, loss, ws, stream=None):
    return load().rsvd_mlp_grad(h, batch, _ptr(X), _ptr(yl), _ptr(yq), lam, _ptr(theta), _ptr(grad), _ptr(loss),
                                _ptr(ws), ws.numel() if ws is not None else 0, _stream(stream))


def rsvd_mlp_train_step(h, batch, X, yl, yq, lam, theta, m1, m2, step, lr, loss, ws, stream=None):
    return load().rsvd_mlp_train_step(h, batch, _ptr(X), _ptr(yl), _ptr(yq), lam, _ptr(theta), _ptr(m1), _ptr(m2),
                                      step, lr, _ptr(loss), _ptr(ws), ws.numel() if ws is not None else 0,
                                      _stream(stream))


def rsvd_controller_attach(h, theta, quantile=0.9, safety=0.8):
    return load().rsvd_controller_attach(h, _ptr(theta), quantile, safety)


def rsvd_controller_last(h):
    info = (ctypes.c_int * 5)()
    est = (ctypes.c_double * 2)()
    _check(load().rsvd_controller_last(h, info, est), h)
    return {"l": info[0], "q": info[1], "accepted": bool(info[2]), "fallback": info[3] == 1,
            "escalated": info[3] == 2, "rank": info[4], "est_rel": est[0], "spec_bound_rel": est[1]}


def rsvd_controller_fallback(h, mode):
    return _check(load().rsvd_controller_fallback(h, int(mode)), h)


def rsvd_kernel_launches(h):
    out = ctypes.c_longlong()
    _check(load().rsvd_kernel_launches(h, ctypes.byref(out)), h)
    return out.value


def rsvd_profile(h, on):
    return _check(load().rsvd_profile(h, int(on)), h)


def rsvd_profile_read(h, kind):
    ms = ctypes.c_double()
    cnt = ctypes.c_longlong()
    _check(load().rsvd_profile_read(h, kind, ctypes.byref(ms), ctypes.byref(cnt)), h)
    return ms.value, cnt.value


# -------------------------------------------------------------- convenience --
def make_params(k, p=10, q=1, seed=0, prec=RSVD_F32, flags=0, tol=0.0, block=16, max_rank=0):
    return Params(k=k, p=p, q=q, block=block, max_rank=max_rank, probe_cols=0, tol=tol, seed=seed, prec=prec,
                  flags=flags)


def _prec_dtype(prec):
    import torch
    return torch.float64 if prec == RSVD_F64 else torch.float32


def fixed_rank(A, k, p=10, q=1, seed=0, prec=RSVD_F32, full=False, sync=True, ws=None, out=None, centre=False,
               krylov=False, single_pass=False, symmetric=False, srft=False):
    """A ~= U diag(D) V^T by rsvd_fixed_rank.  A: (m, n) row-major CUDA tensor
    (float64 for RSVD_F64, else float32).  centre=True factors the
    column-centred matrix without forming it (RSVD_FLAG_CENTER);
    krylov=True takes the block Krylov basis of q blocks (RSVD_FLAG_KRYLOV);
    single_pass=True is the single-pass SVD (q must be 0), with
    symmetric=True the single-pass EVD (D signed, V = U); srft=True takes
    the SRFT test matrix (q must be 0; U and V come back complex).  Returns
    (U, D, V)."""
    import torch
    h = handle(A.device.index)
    m, n = A.shape
    flags = (RSVD_FLAG_RETURN_FULL_L if full else 0) | (RSVD_FLAG_SYNC if sync else 0)
    flags |= (RSVD_FLAG_CENTER if centre else 0) | (RSVD_FLAG_KRYLOV if krylov else 0)
    flags |= (RSVD_FLAG_SINGLE_PASS if single_pass else 0) | (RSVD_FLAG_SYMMETRIC if symmetric else 0)
    flags |= RSVD_FLAG_SRFT if srft else 0
    prm = make_params(k, p, q, seed, prec, flags)
    kk = ((k + p) * (q if krylov else 1)) if full else k
    dt = _prec_dtype(prec)
    if srft:
        dt = torch.complex128 if prec == RSVD_F64 else torch.complex64
    if out is None:
        U = torch.empty(m, kk, dtype=dt, device=A.device)
        D = torch.empty(kk, dtype=torch.float64, device=A.device)
        V = torch.empty(n, kk, dtype=dt, device=A.device)
    else:
        U, D, V = out
    if ws is None:
        ws = _empty_ws(rsvd_workspace_size(h, m, n, prm), A.device)
    _check(rsvd_fixed_rank(h, m, n, A, A.stride(0), prm, U, U.stride(0), D, V, V.stride(0), ws), h)
    return U, D, V


def adaptive_tol(A, tol, block=16, max_rank=0, seed=0, prec=RSVD_F32, q=0, controller=False, spectral=False):
    """Tolerance-driven randomized SVD by rsvd_adaptive_tol (q power steps per
    block; with controller=True the learned controller attached to the
    device's handle chooses (l, q); with spectral=True tol is an absolute
    spectral-norm tolerance, RSVD_FLAG_SPECTRAL).  Returns (U, D, V, rank,
    err, status): U, V have max_rank columns, the first `rank` valid; status
    is RSVD_OK or RSVD_E_NOT_CONVERGED (other failures raise)."""
    import torch
    h = handle(A.device.index)
    m, n = A.shape
    flags = (RSVD_FLAG_USE_CONTROLLER if controller else 0) | (RSVD_FLAG_SPECTRAL if spectral else 0)
    prm = make_params(0, 0, q, seed, prec, flags, tol=tol, block=block, max_rank=max_rank)
    R = max_rank if max_rank > 0 else min(m, n, 128 if prec == RSVD_F64 else 256)
    dt = _prec_dtype(prec)
    U = torch.empty(m, R, dtype=dt, device=A.device)
    D = torch.empty(R, dtype=torch.float64, device=A.device)
    V = torch.empty(n, R, dtype=dt, device=A.device)
    rank = torch.zeros(1, dtype=torch.int32, device=A.device)
    err = torch.zeros(1, dtype=torch.float64, device=A.device)
    ws = _empty_ws(rsvd_workspace_size(h, m, n, prm), A.device)
    code = rsvd_adaptive_tol(h, m, n, A, A.stride(0), prm, U, U.stride(0), D, V, V.stride(0), rank, err, ws)
    if code not in (RSVD_OK, RSVD_E_NOT_CONVERGED):
        raise RsvdError(code, last_error(h))
    return U, D, V, int(rank.item()), float(err.item()), code


class BatchPlan:
    """Device-resident arguments and outputs of one rsvd_batched call.

    The count problems' matrices live in one float32 buffer ``A`` (block p at
    an offset that is a multiple of 4 elements, row-major with lda = n); the
    outputs in ``U`` (m x R blocks), ``V`` (n x R blocks) and ``D`` (count x R
    doubles).  The device arrays of sizes and pointers are built once, so a
    plan can be run many times and captured into a CUDA graph."""

    def __init__(self, shapes, R=64, device="cuda"):
        import torch
        self.count, self.R, self.shapes = len(shapes), int(R), [(int(a), int(b)) for a, b in shapes]
        up4 = lambda x: (x + 3) // 4 * 4
        self.a_off, self.u_off, self.v_off = [], [], []
        ta = tu = tv = 0
        for m, n in self.shapes:
            self.a_off.append(ta)
            self.u_off.append(tu)
            self.v_off.append(tv)
            ta, tu, tv = ta + up4(m * n), tu + up4(m * R), tv + up4(n * R)
        f32 = torch.float32
        self.A = torch.zeros(max(ta, 4), dtype=f32, device=device)
        self.U = torch.empty(max(tu, 4), dtype=f32, device=device)
        self.V = torch.empty(max(tv, 4), dtype=f32, device=device)
        self.D = torch.empty(max(self.count * R, 1), dtype=torch.float64, device=device)
        i32, i64 = torch.int32, torch.int64
        self.m = torch.tensor([s[0] for s in self.shapes] or [0], dtype=i32, device=device)
        self.n = torch.tensor([s[1] for s in self.shapes] or [0], dtype=i32, device=device)
        self.lda = self.n.clone()
        base = lambda t, offs, es: torch.tensor([t.data_ptr() + es * o for o in offs] or [0], dtype=i64,
                                                device=device)
        self.a_ptr = base(self.A, self.a_off, 4)
        self.u_ptr = base(self.U, self.u_off, 4)
        self.v_ptr = base(self.V, self.v_off, 4)
        self.d_ptr = base(self.D, [p * R for p in range(self.count)], 8)
        self.rank = torch.zeros(max(self.count, 1), dtype=i32, device=device)
        self.err = torch.zeros(max(self.count, 1), dtype=torch.float64, device=device)
        self.status = torch.zeros(max(self.count, 1), dtype=i32, device=device)
        self.ws = None

    def block(self, p):
        m, n = self.shapes[p]
        return self.A[self.a_off[p]:self.a_off[p] + m * n].view(m, n)

    def result(self, p):
        """(U, D, V) views of problem p: m x R, R, n x R."""
        m, n = self.shapes[p]
        R = self.R
        return (self.U[self.u_off[p]:self.u_off[p] + m * R].view(m, R), self.D[p * R:(p + 1) * R],
                self.V[self.v_off[p]:self.v_off[p] + n * R].view(n, R))


def batched_run(plan, tol, block=16, seed=0, flags=0, stream=None):
    """Enqueue rsvd_batched for a BatchPlan; returns the call's status (with
    RSVD_FLAG_SYNC in flags, the first device-side failure)."""
    h = handle(plan.A.device.index)
    prm = make_params(0, 0, 0, seed, RSVD_F32, flags, tol=tol, block=block, max_rank=plan.R)
    if plan.ws is None:
        plan.ws = _empty_ws(rsvd_batched_workspace_size(h, plan.count, prm), plan.A.device)
    return rsvd_batched(h, plan.count, plan.m, plan.n, plan.a_ptr, plan.lda, prm, plan.u_ptr, plan.d_ptr,
                        plan.v_ptr, plan.rank, plan.err, plan.status, plan.ws, stream)


def batched_autotune(plan, tol, block=16, seed=0, stream=None):
    """Time every launch variant of rsvd_batched on a BatchPlan and keep the
    fastest for this device's handle.  Returns (variant, per-variant ms)."""
    h = handle(plan.A.device.index)
    prm = make_params(0, 0, 0, seed, RSVD_F32, 0, tol=tol, block=block, max_rank=plan.R)
    if plan.ws is None:
        plan.ws = _empty_ws(rsvd_batched_workspace_size(h, plan.count, prm), plan.A.device)
    code, var, ms = rsvd_batched_autotune(h, plan.count, plan.m, plan.n, plan.a_ptr, plan.lda, prm, plan.u_ptr,
                                          plan.d_ptr, plan.v_ptr, plan.rank, plan.err, plan.status, plan.ws, stream)
    if code not in (RSVD_OK, RSVD_E_NOT_CONVERGED, RSVD_E_INVALID, RSVD_E_BREAKDOWN, RSVD_E_NONFINITE):
        raise RsvdError(code, last_error(h))
    return var, ms


def batched(blocks, tol, block=16, max_rank=64, seed=0):
    """Solve a list of float32 CUDA matrices by rsvd_batched.  Returns
    (plan, code): plan.result(p), plan.rank, plan.err and plan.status hold
    the per-problem outputs."""
    plan = BatchPlan([tuple(b.shape) for b in blocks], R=max_rank, device=blocks[0].device if blocks else "cuda")
    for p, b in enumerate(blocks):
        plan.block(p).copy_(b)
    code = batched_run(plan, tol, block=block, seed=seed, flags=RSVD_FLAG_SYNC)
    if code not in (RSVD_OK, RSVD_E_NOT_CONVERGED, RSVD_E_INVALID, RSVD_E_BREAKDOWN, RSVD_E_NONFINITE):
        raise RsvdError(code, last_error(handle(plan.A.device.index)))
    return plan, code


def gaussian(n, l, seed, stream_id=0, col0=0, dtype=None, device="cuda"):
    import torch
    dtype = torch.float32 if dtype is None else dtype
    code = {torch.float64: RSVD_DT_F64, torch.float32: RSVD_DT_F32, torch.bfloat16: RSVD_DT_BF16}[dtype]
    out = torch.empty(n, l, dtype=dtype, device=device)
    h = handle(out.device.index)
    _check(rsvd_gaussian(h, n, l, seed, stream_id, col0, code, out, l), h)
    return out


def philox_words(n_groups, l, seed, stream_id=0, col0=0, device="cuda"):
    import torch
    out = torch.empty(l * n_groups * 4, dtype=torch.int32, device=device)
    h = handle(out.device.index)
    _check(rsvd_philox_words(h, n_groups, l, seed, stream_id, col0, out), h)
    return out


def sketch(A, X, trans=False, prec=RSVD_F32):
    """Y = A X (trans=False) or A^T X (trans=True) through rsvd_sketch."""
    import torch
    h = handle(A.device.index)
    m, n = A.shape
    l = X.shape[1]
    M = n if trans else m
    ydt = torch.float64 if prec == RSVD_F64 else torch.float32
    Y = torch.empty(M, l, dtype=ydt, device=A.device)
    ws = _empty_ws(rsvd_sketch_workspace_size(h, prec, int(trans), m, n, l), A.device)
    _check(rsvd_sketch(h, prec, int(trans), m, n, l, A, A.stride(0), X, X.stride(0), Y, Y.stride(0), ws), h)
    return Y


def project(A, Q, prec=RSVD_F32):
    """B^T = A^T Q through rsvd_project."""
    import torch
    h = handle(A.device.index)
    m, n = A.shape
    l = Q.shape[1]
    Bt = torch.empty(n, l, dtype=torch.float64 if prec == RSVD_F64 else torch.float32, device=A.device)
    ws = _empty_ws(rsvd_project_workspace_size(h, prec, m, n, l), A.device)
    _check(rsvd_project(h, prec, m, n, l, A, A.stride(0), Q, Q.stride(0), Bt, Bt.stride(0), ws), h)
    return Bt


def orth(Y, prec=RSVD_F32, want_r=True):
    """Q, R with Y = Q R through rsvd_orth (Y is copied, not overwritten)."""
    import torch
    h = handle(Y.device.index)
    rows, l = Y.shape
    Q = Y.clone()
    R = torch.empty(l, l, dtype=torch.float64, device=Y.device) if want_r else None
    ws = _empty_ws(rsvd_orth_workspace_size(h, prec, rows, l), Y.device)
    _check(rsvd_orth(h, prec, rows, l, Q, Q.stride(0), R, ws), h)
    st = rsvd_query_status(h, ws)
    if st != RSVD_OK:
        raise RsvdError(st, "orth device status")
    return Q, R


# ----------------------------------------------------- learned controller --
def probe_features(A, seed=0):
    """(features (17 floats, CUDA tensor), ||A||_F^2) of a float32 CUDA matrix."""
    import torch
    h = handle(A.device.index)
    m, n = A.shape
    feat = torch.empty(CTRL_D_IN, dtype=torch.float32, device=A.device)
    fro2 = torch.empty(1, dtype=torch.float64, device=A.device)
    ws = _empty_ws(rsvd_probe_workspace_size(h, m, n), A.device)
    _check(rsvd_probe_features(h, m, n, A, A.stride(0), seed, feat, fro2, ws), h)
    return feat, fro2


def mlp_forward(X, theta):
    import torch
    h = handle(X.device.index)
    logits = torch.empty(X.shape[0], CTRL_OUT, dtype=torch.float32, device=X.device)
    _check(rsvd_mlp_forward(h, X.shape[0], X, theta, logits), h)
    return logits


def mlp_grad(X, yl, yq, lam, theta):
    import torch
    h = handle(X.device.index)
    grad = torch.empty(CTRL_PARAMS, dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float64, device=X.device)
    ws = _empty_ws(rsvd_mlp_workspace_size(h, X.shape[0]), X.device)
    _check(rsvd_mlp_grad(h, X.shape[0], X, yl, yq, lam, theta, grad, loss, ws), h)
    return grad, loss


class Trainer:
    """Adam training of the controller network on the GPU through
    rsvd_mlp_train_step.  theta (float32 CUDA tensor of CTRL_PARAMS) is
    updated in place."""

    def __init__(self, theta, lr=1e-3, lam=0.5):
        import torch
        self.theta, self.lr, self.lam = theta, float(lr), float(lam)
        self.m1 = torch.zeros_like(theta)
        self.m2 = torch.zeros_like(theta)
        self.t = 0
        self.h = handle(theta.device.index)
        self.ws = None
        self.loss = torch.zeros(1, dtype=torch.float64, device=theta.device)

    def step(self, X, yl, yq):
        if self.ws is None or self.ws.numel() < rsvd_mlp_workspace_size(self.h, X.shape[0]):
            self.ws = _empty_ws(rsvd_mlp_workspace_size(self.h, X.shape[0]), X.device)
        self.t += 1
        _check(rsvd_mlp_train_step(self.h, X.shape[0], X, yl, yq, self.lam, self.theta, self.m1, self.m2, self.t,
                                   self.lr, self.loss, self.ws), self.h)
        return self.loss


L_STEP = 16
N_L_CLASSES = 16


def label_from_ranks(ranks, converged):
    """Training label (l class, q) from the adaptive ranks l_q, q = 0..3: the q
    that meets the tolerance with the least sketch work (2q + 2) l_q, ties to
    the smaller q; (15, 2) when none met it."""
    best = None
    for q, (r, ok) in enumerate(zip(ranks, converged)):
        if ok and (best is None or (2 * q + 2) * r < best[0]):
            best = ((2 * q + 2) * r, q, r)
    if best is None:
        return N_L_CLASSES - 1, 2
    _, q, r = best
    return min(max((r + L_STEP - 1) // L_STEP - 1, 0), N_L_CLASSES - 1), q


def adaptive_labels(A, tol, seed=0, max_rank=256, block=16):
    """Ranks l_q of rsvd_adaptive_tol (binary32, power steps q = 0..3) and the
    label they give."""
    ranks, conv = [], []
    for q in range(4):
        _, _, _, r, _, code = adaptive_tol(A, tol, block=block, max_rank=max_rank, seed=seed, q=q)
        ranks.append(r)
        conv.append(code == RSVD_OK)
    return ranks, conv, label_from_ranks(ranks, conv)
