"""Thin Python binding of libtgba.so (include/tgba.h), with the C names.

Argument marshalling only: every step runs in the library's CUDA kernels (and its cuSOLVER /
cuBLAS calls).  Device buffers are torch CUDA tensors allocated by the caller; streams default
to torch's current stream.  There is no fallback: if the library is not built or cannot be
loaded, the first call raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

TGBA_OK, TGBA_EINVAL, TGBA_ENOMEM, TGBA_ECUDA, TGBA_ENUMERIC, TGBA_ETIMEOUT, TGBA_ELIMIT = range(7)
_NAMES = {0: "TGBA_OK", 1: "TGBA_EINVAL", 2: "TGBA_ENOMEM", 3: "TGBA_ECUDA", 4: "TGBA_ENUMERIC",
          5: "TGBA_ETIMEOUT", 6: "TGBA_ELIMIT"}

# every symbol include/tgba.h declares
SYMBOLS = ("tgba_last_error", "tgba_device_count", "tgba_build_basis", "tgba_basis_info", "tgba_basis_totals",
           "tgba_basis_free", "tgba_compute_x", "tgba_x_stats", "tgba_x_export", "tgba_x_pairs", "tgba_x_direct", "tgba_z_elements", "tgba_table",
           "tgba_assemble_heff", "tgba_eigvals", "tgba_eigvals_ex", "tgba_eigvals_wait_check", "tgba_dsf", "tgba_dsf_k", "tgba_quench", "tgba_quench_ordered", "tgba_quench_correlators", "tgba_screen_create",
           "tgba_screen_nparams", "tgba_screen_params", "tgba_screen_grad", "tgba_screen_train",
           "tgba_screen_predict", "tgba_screen_free", "tgba_table_noalloc", "tgba_dgemm_tc", "tgba_profile", "tgba_fp64_peak")


class TgbaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_NAMES.get(code, code), msg))
        self.code = code


class _Model(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("J", ctypes.c_double), ("h_z", ctypes.c_double), ("h_x", ctypes.c_double)]


class _Trunc(ctypes.Structure):
    _fields_ = [("max_qp", ctypes.c_int32), ("e_cut", ctypes.c_double), ("max_per_parity", ctypes.c_int64)]


class _Prof(ctypes.Structure):
    _fields_ = [("table_ms", ctypes.c_double), ("pfaffian_ms", ctypes.c_double), ("pfaffian_flops", ctypes.c_double),
                ("pfaffian_launches", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("upload_bytes", ctypes.c_int64), ("evaluated", ctypes.c_int64),
                ("tune_mode", ctypes.c_int32), ("tune_threads", ctypes.c_int32), ("tune_ms", ctypes.c_double * 8),
                ("tridiag_ms", ctypes.c_double), ("bisect_ms", ctypes.c_double), ("tridiag_flops", ctypes.c_double),
                ("eig_matrices", ctypes.c_int64), ("eig_cluster", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("quench_ms", ctypes.c_double), ("quench_flops", ctypes.c_double), ("quench_terms", ctypes.c_int64),
                ("quench_prep_ms", ctypes.c_double), ("quench_gram_ms", ctypes.c_double),
                ("quench_eval_ms", ctypes.c_double)]


_lib = None
_P, _I32, _I64, _D, _VP = ctypes.POINTER, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


def lib():
    """Load libtgba.so (built in-tree by paper_2410_04204_gb300/build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libtgba.so is not built (%s); run paper_2410_04204_gb300.build.build()" % _build.LIB)
        L = ctypes.CDLL(_build.LIB)
        sig = {
            "tgba_last_error": (ctypes.c_char_p, []),
            "tgba_device_count": (_I32, []),
            "tgba_build_basis": (_I32, [_P(_Model), _P(_I32), _I32, _P(_Trunc), _P(_VP)]),
            "tgba_basis_info": (_I32, [_VP, _I32, _P(_I64), _P(_I64), _VP, _VP, _VP, _VP]),
            "tgba_basis_totals": (_I32, [_VP, _P(_I32), _P(_I64), _P(_I64)]),
            "tgba_basis_free": (_I32, [_VP]),
            "tgba_compute_x": (_I32, [_VP, _VP, _D, _D, _VP]),
            "tgba_x_stats": (_I32, [_VP, _P(_I64), _P(_I64)]),
            "tgba_x_export": (_I32, [_VP, _I32, _VP, _VP]),
            "tgba_x_pairs": (_I32, [_VP, _I32, _VP, _I64, _VP, _VP]),
            "tgba_x_direct": (_I32, [_VP, _I32, _VP, _I64, _VP, _VP]),
            "tgba_z_elements": (_I32, [_VP, _I32, _I32, _I32, _VP, _I64, _VP, _VP]),
            "tgba_table": (_I32, [_VP, _VP, _VP, _VP]),
            "tgba_assemble_heff": (_I32, [_VP, _D, _VP, _D, _VP, _VP]),
            "tgba_eigvals": (_I32, [_VP, _VP, _I32, _VP, _VP]),
            "tgba_eigvals_ex": (_I32, [_VP, _VP, _I32, _I32, _VP, _VP]),
            "tgba_eigvals_wait_check": (_I32, [_VP, _VP, _I32, ctypes.c_uint32, _I32, _I32, _VP, _VP]),
            "tgba_dsf": (_I32, [_VP, _I32, _D, _D, _D, _I32, _D, _VP, _VP, _I32, _VP, _VP, _VP]),
            "tgba_dsf_k": (_I32, [_VP, _I32, _I32, _D, _D, _D, _I32, _D, _VP, _VP, _I32, _VP, _VP, _VP]),
            "tgba_quench": (_I32, [_VP, _I32, _D, _VP, _VP, _I32, _D, _I32, _I32, _VP, _VP, _VP, _VP]),
            "tgba_quench_ordered": (_I32, [_VP, _I32, _D, _VP, _VP, _I32, _I32, _D, _I32, _I32, _VP, _VP, _VP, _VP,
                                           _VP]),
            "tgba_quench_correlators": (_I32, [_VP, _I32, _D, _D, _D, _I32, _D, _I32, _I32, _VP, _VP, _VP, _VP,
                                               _VP]),
            "tgba_screen_create": (_I32, [_I32, _VP, ctypes.c_uint64, _P(_VP)]),
            "tgba_screen_nparams": (_I32, [_VP, _P(_I64)]),
            "tgba_screen_params": (_I32, [_VP, _VP]),
            "tgba_screen_grad": (_I32, [_VP, _VP, _VP, _I64, _VP, _P(_D), _VP]),
            "tgba_screen_train": (_I32, [_VP, _I32, _I64, ctypes.c_uint64, _I32, _I32, _P(_VP), _VP, _VP]),
            "tgba_screen_predict": (_I32, [_VP, _VP, _I32, _VP, _VP]),
            "tgba_screen_free": (_I32, [_VP]),
            "tgba_table_noalloc": (_I32, [_I32, _D, _D, _VP, _VP, _VP]),
            "tgba_dgemm_tc": (_I32, [_I32, _I32, _I32, _VP, _I64, _VP, _I64, _VP, _I64, _VP]),
            "tgba_profile": (_I32, [_VP, _P(_Prof)]),
            "tgba_fp64_peak": (_I32, [_I32, _P(_D)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code):
    if code != TGBA_OK:
        raise TgbaError(code, lib().tgba_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _cuda_tensor(t, dtype, numel=None, name="buffer"):
    import torch
    if t is None:
        return
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError("%s must be a contiguous CUDA %s tensor" % (name, dtype))
    if numel is not None and t.numel() < numel:
        raise ValueError("%s holds %d elements, needs %d" % (name, t.numel(), numel))


def tgba_device_count():
    return int(lib().tgba_device_count())


def tgba_build_basis(L, h_z, sectors, max_qp, e_cut=-1.0, max_per_parity=0, J=1.0):
    """Returns the basis handle (int)."""
    m = _Model(int(L), float(J), float(h_z), 0.0)
    t = _Trunc(int(max_qp), -1.0 if e_cut is None else float(e_cut), int(max_per_parity or 0))
    sec = np.ascontiguousarray(np.asarray(list(sectors), dtype=np.int32))
    h = _VP()
    _check(lib().tgba_build_basis(ctypes.byref(m), sec.ctypes.data_as(_P(_I32)), len(sec), ctypes.byref(t),
                                  ctypes.byref(h)))
    _MAX_QP[h.value] = int(max_qp)
    return h.value


_MAX_QP = {}     # handle -> max_qp, the row length of the modes table tgba_basis_info writes


def tgba_basis_info(b, s, max_qp=None):
    """Sizes and state tables of sector s (numpy, basis order).  The modes table has the basis's
    max_qp columns; a different max_qp argument is an error."""
    mq = _MAX_QP.get(b, max_qp)
    if mq is None or (max_qp is not None and max_qp != mq):
        raise ValueError("max_qp must be the basis's own (%s)" % mq)
    max_qp = mq
    n_ns, n_r = _I64(), _I64()
    _check(lib().tgba_basis_info(b, s, ctypes.byref(n_ns), ctypes.byref(n_r), None, None, None, None))
    n = n_ns.value + n_r.value
    E = np.zeros(n, np.float64)
    par = np.zeros(n, np.uint8)
    nqp = np.zeros(n, np.uint8)
    modes = np.zeros((n, max(1, max_qp)), np.int16)
    _check(lib().tgba_basis_info(b, s, ctypes.byref(n_ns), ctypes.byref(n_r), E.ctypes.data, par.ctypes.data,
                                 nqp.ctypes.data, modes.ctypes.data))
    return dict(n_ns=n_ns.value, n_r=n_r.value, E0=E, parity=par, nqp=nqp, modes=modes[:, :max_qp])


def tgba_sector_sizes(b):
    """[(n_ns, n_r)] of every sector, in order."""
    out = []
    for s in range(tgba_basis_totals(b)[0]):
        n_ns, n_r = _I64(), _I64()
        _check(lib().tgba_basis_info(b, s, ctypes.byref(n_ns), ctypes.byref(n_r), None, None, None, None))
        out.append((n_ns.value, n_r.value))
    return out


def _n_states(b):
    return sum(a + c for a, c in tgba_sector_sizes(b))


def tgba_basis_totals(b):
    ns, ne, nh = _I32(), _I64(), _I64()
    _check(lib().tgba_basis_totals(b, ctypes.byref(ns), ctypes.byref(ne), ctypes.byref(nh)))
    return ns.value, ne.value, nh.value


def tgba_basis_free(b):
    _check(lib().tgba_basis_free(b))
    _MAX_QP.pop(b, None)


def tgba_compute_x(b, screen=None, screen_tau=0.0, screen_hx=0.0, stream=None):
    _check(lib().tgba_compute_x(b, screen, float(screen_tau), float(screen_hx), _stream(stream)))


def tgba_x_stats(b):
    ev, sc = _I64(), _I64()
    _check(lib().tgba_x_stats(b, ctypes.byref(ev), ctypes.byref(sc)))
    return ev.value, sc.value


def tgba_x_export(b, s, x_out, stream=None):
    """x_out: complex128 CUDA tensor with n_ns * n_r elements."""
    import torch
    _cuda_tensor(x_out, torch.complex128, name="x_out")
    _check(lib().tgba_x_export(b, s, _ptr(x_out), _stream(stream)))


def tgba_x_pairs(b, s, pairs, out, stream=None):
    """pairs: int32 CUDA tensor [n, 2] (NS index, R index); out: complex128 CUDA tensor [n]."""
    import torch
    _cuda_tensor(pairs, torch.int32, name="pairs")
    _cuda_tensor(out, torch.complex128, pairs.shape[0], name="out")
    _check(lib().tgba_x_pairs(b, s, _ptr(pairs), pairs.shape[0], _ptr(out), _stream(stream)))


def tgba_x_direct(b, s, pairs, out, stream=None):
    """pairs: int32 CUDA tensor [n, 2] (NS index, R index); out: complex128 CUDA tensor [n]."""
    import torch
    _cuda_tensor(pairs, torch.int32, name="pairs")
    _cuda_tensor(out, torch.complex128, pairs.shape[0], name="out")
    _check(lib().tgba_x_direct(b, s, _ptr(pairs), pairs.shape[0], _ptr(out), _stream(stream)))


def tgba_z_elements(b, s, parity, j, pairs, out, stream=None):
    """<phi_a| sigma^x_1 sigma^x_{j+1} |phi_b> for states of one parity (0 NS, 1 R) of sector s.
    pairs: int32 CUDA tensor [n, 2] (state indices of that parity); out: complex128 CUDA tensor [n]."""
    import torch
    _cuda_tensor(pairs, torch.int32, name="pairs")
    _cuda_tensor(out, torch.complex128, pairs.shape[0], name="out")
    _check(lib().tgba_z_elements(b, s, parity, j, _ptr(pairs), pairs.shape[0], _ptr(out), _stream(stream)))


def tgba_table(b, table_out=None, stream=None):
    """Returns C0 (complex); fills table_out (float64 CUDA tensor, 2L x 2L) if given."""
    import torch
    _cuda_tensor(table_out, torch.float64, name="table_out")
    c0 = np.zeros(2)
    _check(lib().tgba_table(b, c0.ctypes.data, _ptr(table_out), _stream(stream)))
    return complex(c0[0], c0[1])


def tgba_assemble_heff(b, h_x, heff_out, screen=None, screen_tau=0.0, stream=None):
    """heff_out: complex128 CUDA tensor with n_heff elements (all sectors, column-major each)."""
    import torch
    _cuda_tensor(heff_out, torch.complex128, name="heff_out")
    _check(lib().tgba_assemble_heff(b, float(h_x), screen, float(screen_tau), _ptr(heff_out), _stream(stream)))


def tgba_eigvals(b, h_x, evals_out, stream=None, method=0):
    """h_x: one field or a list; evals_out: float64 CUDA tensor [len(h_x) * n_states].
    method: 0 automatic, 1 native (tridiagonalisation + bisection), 2 cuSOLVER."""
    import torch
    hx = np.ascontiguousarray(np.atleast_1d(np.asarray(h_x, np.float64)))
    _cuda_tensor(evals_out, torch.float64, len(hx) * _n_states(b), name="evals_out")
    _check(lib().tgba_eigvals_ex(b, hx.ctypes.data, len(hx), int(method), _ptr(evals_out), _stream(stream)))


def tgba_eigvals_wait_check(b, h_x, evals_out, spin_limit, withhold_matrix=-1, withhold_rank=0, stream=None):
    """The native solver with a short wait limit and, optionally, one CTA withheld from its
    group (failure-detection check of the bounded waits)."""
    import torch
    hx = np.ascontiguousarray(np.atleast_1d(np.asarray(h_x, np.float64)))
    _cuda_tensor(evals_out, torch.float64, len(hx) * _n_states(b), name="evals_out")
    _check(lib().tgba_eigvals_wait_check(b, hx.ctypes.data, len(hx), int(spin_limit), int(withhold_matrix),
                                         int(withhold_rank), _ptr(evals_out), _stream(stream)))


def tgba_dsf(b, s, h_x, w_min, w_max, n_w, eta, S_out, evals_out=None, n_ev=0, weights_out=None, dE_out=None,
             stream=None):
    import torch
    _cuda_tensor(S_out, torch.float32, n_w, name="S_out")
    for t in (evals_out, weights_out, dE_out):
        _cuda_tensor(t, torch.float64)
    _check(lib().tgba_dsf(b, s, float(h_x), float(w_min), float(w_max), int(n_w), float(eta), _ptr(S_out),
                          _ptr(evals_out), int(n_ev), _ptr(weights_out), _ptr(dE_out), _stream(stream)))


def tgba_dsf_k(b, s, s0, h_x, w_min, w_max, n_w, eta, S_out, evals_out=None, n_ev=0, weights_out=None, dE_out=None,
               stream=None):
    """S(k, w) at the momentum of sector s; s0 is the k = 0 sector (ground state)."""
    import torch
    _cuda_tensor(S_out, torch.float32, n_w, name="S_out")
    n = 0
    if (weights_out is not None or dE_out is not None) and 0 <= s < tgba_basis_totals(b)[0]:
        n = sum(tgba_sector_sizes(b)[s])
    _cuda_tensor(evals_out, torch.float64, n_ev, name="evals_out")
    _cuda_tensor(weights_out, torch.float64, n, name="weights_out")
    _cuda_tensor(dE_out, torch.float64, n, name="dE_out")
    _check(lib().tgba_dsf_k(b, int(s), int(s0), float(h_x), float(w_min), float(w_max), int(n_w), float(eta),
                            _ptr(S_out), _ptr(evals_out), int(n_ev), _ptr(weights_out), _ptr(dE_out), _stream(stream)))


def tgba_quench(b, s, h_z0, hx_variants, ecut_variants, t_max, n_t, mx_out, norm_out=None, method=0, stream=None):
    """Returns the retained basis size of each variant (method: 0 automatic, 1 eigen, 2 Chebyshev)."""
    import torch
    hx = np.ascontiguousarray(np.asarray(hx_variants, np.float64))
    ec = np.ascontiguousarray(np.asarray(ecut_variants, np.float64))
    if hx.shape != ec.shape:
        raise ValueError("one cutoff per h_x variant")
    _cuda_tensor(mx_out, torch.float64, len(hx) * n_t, name="mx_out")
    _cuda_tensor(norm_out, torch.float64, len(hx), name="norm_out")
    chi = np.zeros(len(hx), np.int64)
    _check(lib().tgba_quench(b, s, float(h_z0), hx.ctypes.data, ec.ctypes.data, len(hx), float(t_max), int(n_t),
                             int(method), _ptr(mx_out), _ptr(norm_out), chi.ctypes.data, _stream(stream)))
    return chi


def tgba_quench_ordered(b, s, h_z0, hx_variants, trunc_variants, order, t_max, n_t, mx_out, norm_out=None,
                        eps_out=None, method=0, stream=None):
    """Quench with energy- (order 0) or overlap-ordered (order 1) nested truncations; eps_out
    (float64 CUDA tensor, len - 1) receives the Eq. 11 metric between successive variants.
    Returns the retained basis size of each variant."""
    import torch
    hx = np.ascontiguousarray(np.asarray(hx_variants, np.float64))
    tr = np.ascontiguousarray(np.asarray(trunc_variants, np.float64))
    if hx.shape != tr.shape:
        raise ValueError("one truncation per h_x variant")
    _cuda_tensor(mx_out, torch.float64, len(hx) * n_t, name="mx_out")
    _cuda_tensor(norm_out, torch.float64, len(hx), name="norm_out")
    _cuda_tensor(eps_out, torch.float64, max(0, len(hx) - 1), name="eps_out")
    chi = np.zeros(len(hx), np.int64)
    _check(lib().tgba_quench_ordered(b, s, float(h_z0), hx.ctypes.data, tr.ctypes.data, len(hx), int(order),
                                     float(t_max), int(n_t), int(method), _ptr(mx_out), _ptr(norm_out),
                                     _ptr(eps_out), chi.ctypes.data, _stream(stream)))
    return chi


def tgba_quench_correlators(b, s, h_z0, h_x, trunc, order, t_max, n_t, j_max, mx_out, corr_out, norm_out=None,
                            stream=None):
    """<sigma^x_1 sigma^x_{j+1}>(t) - <sigma^x>(t)^2, j = 1..j_max, for one truncated quench.
    Returns the kept basis size."""
    import torch
    _cuda_tensor(mx_out, torch.float64, n_t, name="mx_out")
    _cuda_tensor(corr_out, torch.float64, j_max * n_t, name="corr_out")
    _cuda_tensor(norm_out, torch.float64, 1, name="norm_out")
    chi = np.zeros(1, np.int64)
    _check(lib().tgba_quench_correlators(b, s, float(h_z0), float(h_x), float(trunc), int(order), float(t_max),
                                         int(n_t), int(j_max), _ptr(mx_out), _ptr(corr_out), _ptr(norm_out),
                                         chi.ctypes.data, _stream(stream)))
    return int(chi[0])


def tgba_screen_create(width=256, params=None, seed=0):
    """params: float32 numpy array of tgba_screen_nparams entries, or None for a seeded init."""
    h = _VP()
    p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
    _check(lib().tgba_screen_create(int(width), None if p is None else p.ctypes.data, int(seed), ctypes.byref(h)))
    return h.value


def tgba_screen_nparams(s):
    n = _I64()
    _check(lib().tgba_screen_nparams(s, ctypes.byref(n)))
    return n.value


def tgba_screen_params(s):
    out = np.zeros(tgba_screen_nparams(s), np.float32)
    _check(lib().tgba_screen_params(s, out.ctypes.data))
    return out


def tgba_screen_grad(s, x, t, grad_out, stream=None):
    """x: float32 CUDA [B, 20], t: float32 CUDA [B], grad_out: float32 CUDA [nparams]; returns the loss."""
    import torch
    for name, v in (("x", x), ("t", t), ("grad_out", grad_out)):
        _cuda_tensor(v, torch.float32, name=name)
    loss = _D()
    _check(lib().tgba_screen_grad(s, _ptr(x), _ptr(t), int(t.shape[0]), _ptr(grad_out), ctypes.byref(loss),
                                  _stream(stream)))
    return loss.value


def tgba_screen_train(bases, n_samples, seed, epochs, width=256, stream=None):
    """Returns (screen handle, dict of training statistics)."""
    arr = (_VP * len(bases))(*bases)
    h = _VP()
    st = np.zeros(4)
    _check(lib().tgba_screen_train(arr, len(bases), int(n_samples), int(seed), int(width), int(epochs), ctypes.byref(h),
                                   st.ctypes.data, _stream(stream)))
    return h.value, dict(train_rmse=st[0], val_rmse=st[1], margin=st[2], seconds=st[3])


def tgba_screen_predict(s, b, sector, pred_out, stream=None):
    import torch
    _cuda_tensor(pred_out, torch.float32, name="pred_out")
    _check(lib().tgba_screen_predict(s, b, int(sector), _ptr(pred_out), _stream(stream)))


def tgba_screen_free(s):
    _check(lib().tgba_screen_free(s))


def tgba_table_noalloc(L, h_z, table_out, c0_out, J=1.0, stream=None):
    """Contraction table and C0 without any device allocation (see include/tgba.h):
    table_out float64 CUDA [2L * 2L], c0_out float64 CUDA [2]."""
    import torch
    _cuda_tensor(table_out, torch.float64, 4 * L * L, name="table_out")
    _cuda_tensor(c0_out, torch.float64, 2, name="c0_out")
    _check(lib().tgba_table_noalloc(int(L), float(J), float(h_z), _ptr(table_out), _ptr(c0_out), _stream(stream)))


def tgba_profile(b):
    """Stage times of the last tgba_compute_x and the handle's counters (dict)."""
    p = _Prof()
    _check(lib().tgba_profile(b, ctypes.byref(p)))
    out = {k: getattr(p, k) for k, _ in _Prof._fields_}
    out["tune_ms"] = list(p.tune_ms)[:7]
    out.pop("pad_")
    return out


def tgba_dgemm_tc(M, N, K, A, lda, B, ldb, C, ldc, stream=None):
    """C = A B^T in FP64 on the tensor cores: A [M][K] (ld lda), B [N][K] (ld ldb), C column-major
    (ld ldc); float64 CUDA tensors."""
    import torch
    for t, name in ((A, "A"), (B, "B"), (C, "C")):
        _cuda_tensor(t, torch.float64, name=name)
    _check(lib().tgba_dgemm_tc(int(M), int(N), int(K), _ptr(A), int(lda), _ptr(B), int(ldb), _ptr(C), int(ldc),
                               _stream(stream)))


def tgba_fp64_peak(reps=5):
    g = _D()
    _check(lib().tgba_fp64_peak(int(reps), ctypes.byref(g)))
    return g.value
