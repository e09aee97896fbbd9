"""ctypes binding of libsbio.so (the C ABI declared in include/sbio.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Device buffers are passed as torch CUDA tensors (raw pointers are
taken from them), streams as torch.cuda.Stream or raw handles.  Importing this
module raises if the compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsbio.so")

SBIO_OK = 0
SBIO_EINVAL = -1
SBIO_EOVERLAP = -2
SBIO_ENOMEM = -3
SBIO_ECUDA = -4
SBIO_ETIMEOUT = -5
SBIO_ENOTSUP = -6
SBIO_PROLATE = 0
SBIO_OBLATE = 1
SBIO_FP64 = 0
SBIO_MIXED = 1
SBIO_PART_SELF = 1
SBIO_PART_NEAR = 2
SBIO_PART_FAR = 4
SBIO_PART_ALL = 7
SBIO_MAX_P = 24

ERRNAMES = {0: "SBIO_OK", -1: "SBIO_EINVAL", -2: "SBIO_EOVERLAP", -3: "SBIO_ENOMEM", -4: "SBIO_ECUDA",
            -5: "SBIO_ETIMEOUT", -6: "SBIO_ENOTSUP"}


class sbio_spheroid(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("A", C.c_double), ("C", C.c_double),
                ("center", C.c_double * 3), ("quat", C.c_double * 4)]


class sbio_options(C.Structure):
    _fields_ = [("p", C.c_int32), ("n_phi", C.c_int32), ("near_factor", C.c_double),
                ("far_upsample", C.c_int32), ("precision", C.c_int32)]


class sbio_request(C.Structure):
    _fields_ = [("op", C.c_int32), ("n_applies", C.c_int32), ("sph", C.c_void_p), ("M", C.c_int32),
                ("flags", C.c_int32), ("opts", sbio_options), ("coef_host", C.c_void_p),
                ("out_host", C.c_void_p)]


SBIO_OP_LAPLACE = 0
SBIO_OP_STOKES = 1

SBIO_COMPLETION_CI = 0
SBIO_COMPLETION_ETA_CI = 1
SBIO_COMPLETION_S = 2
SBIO_COMPLETION_ETA_S = 3


class sbio_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
                ("rel_residual", C.c_double), ("ms", C.c_double)]


class sbio_peaks(C.Structure):
    _fields_ = [("fp32_ffma_tflops", C.c_double), ("fp32_ffma2_tflops", C.c_double), ("rsqrt_per_s", C.c_double),
                ("fp64_dfma_tflops", C.c_double), ("pairmix_pairs_per_s", C.c_double),
                ("pairsmem_pairs_per_s", C.c_double),
                ("sm_clock_mhz", C.c_double), ("sms", C.c_int32), ("reserved", C.c_int32)]


class SbioError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRNAMES.get(code, code)}: {msg}")
        self.code = code


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libsbio.so not built at {LIB_PATH}; run __graft_entry__.build() "
                      "(python -m paper_2506_20809_gb300.build)")

_lib = C.CDLL(LIB_PATH)

_vp = C.c_void_p
_SIGS = {
    "sbio_version": (C.c_char_p, []),
    "sbio_last_error": (C.c_char_p, [_vp]),
    "sbio_launch_count": (C.c_int64, []),
    "sbio_ctx_create": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(_vp)]),
    "sbio_ctx_destroy": (C.c_int, [_vp]),
    "sbio_ctx_mem_used": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "sbio_geom_create": (C.c_int, [_vp, C.POINTER(sbio_spheroid), C.c_int32, C.POINTER(sbio_options), _vp,
                                   C.POINTER(_vp)]),
    "sbio_geom_destroy": (C.c_int, [_vp]),
    "sbio_geom_info": (C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_size_t)]),
    "sbio_geom_nodes": (C.c_int, [_vp, _vp, _vp, _vp]),
    "sbio_geom_setup_times": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]),
    "sbio_geom_near_pairs": (C.c_int, [_vp, _vp, _vp]),
    "sbio_geom_set_precision": (C.c_int, [_vp, C.c_int32]),
    "sbio_geom_enable_timing": (C.c_int, [_vp, C.c_int32]),
    "sbio_geom_set_launch_shape": (C.c_int, [_vp, C.c_int32, C.c_int32]),
    "sbio_geom_set_overlap": (C.c_int, [_vp, C.c_int32]),
    "sbio_geom_set_near_cap": (C.c_int, [_vp, C.c_int32]),
    "sbio_geom_set_tree_near_cap": (C.c_int, [_vp, C.c_int32]),
    "sbio_geom_tree_order_counts": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_int64)]),
    "sbio_geom_get_tree_near_cap": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
    "sbio_geom_get_tuning": (C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "sbio_geom_autotune": (C.c_int, [_vp, _vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_double)]),
    "sbio_geom_phase_times": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]),
    "sbio_apply_laplace": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "sbio_apply_laplace_parts": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_uint32, _vp]),
    "sbio_apply_laplace_host": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "sbio_apply_stokes_sl": (C.c_int, [_vp, _vp, _vp, _vp]),
    "sbio_apply_stokes_sl_host": (C.c_int, [_vp, _vp, _vp, _vp]),
    "sbio_apply_laplace_deriv": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "sbio_forward_transform": (C.c_int, [_vp, _vp, C.c_int32, _vp, _vp]),
    "sbio_solve_dirichlet": (C.c_int, [_vp, _vp, C.c_int32, C.c_double, C.c_int32, C.c_int32, _vp, _vp, _vp,
                                       C.POINTER(sbio_solve_info), _vp]),
    "sbio_solve_neumann": (C.c_int, [_vp, _vp, C.c_double, C.c_int32, C.c_int32, _vp,
                                     C.POINTER(sbio_solve_info), _vp]),
    "sbio_targets_create": (C.c_int, [_vp, _vp, C.c_int64, _vp, C.POINTER(_vp)]),
    "sbio_targets_destroy": (C.c_int, [_vp]),
    "sbio_targets_info": (C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_size_t)]),
    "sbio_eval_targets": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "sbio_eval_targets_deriv": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sbio_apply_laplace_limit": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_int32, _vp]),
    "sbio_apply_stokes_dl_limit": (C.c_int, [_vp, _vp, _vp, C.c_int32, _vp]),
    "sbio_apply_laplace_deriv_limit": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_int32, _vp]),
    "sbio_eval_targets_stokes": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "sbio_eval_targets_stokes_dl": (C.c_int, [_vp, _vp, _vp, _vp]),
    "sbio_apply_stokes_dl": (C.c_int, [_vp, _vp, _vp, _vp]),
    "sbio_geom_set_stokes_tuning": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32]),
    "sbio_geom_get_stokes_tuning": (C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                              C.POINTER(C.c_int32)]),
    "sbio_geom_autotune_stokes": (C.c_int, [_vp, _vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                            C.POINTER(C.c_double)]),
    "sbio_batch_create": (C.c_int, [_vp, C.POINTER(_vp), C.c_int32, C.POINTER(_vp)]),
    "sbio_batch_destroy": (C.c_int, [_vp]),
    "sbio_batch_info": (C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int32)]),
    "sbio_batch_set_far_tt": (C.c_int, [_vp, C.c_int32]),
    "sbio_batch_apply": (C.c_int, [_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), _vp]),
    "sbio_batch_autotune": (C.c_int, [_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), _vp,
                                      C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                      C.POINTER(C.c_double)]),
    "sbio_server_create": (C.c_int, [_vp, C.c_int32, C.c_size_t, C.POINTER(_vp)]),
    "sbio_server_submit": (C.c_int, [_vp, C.POINTER(sbio_request), C.POINTER(C.c_int64)]),
    "sbio_server_wait": (C.c_int, [_vp, C.c_int64, C.c_double, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double)]),
    "sbio_server_stats": (C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int32), C.POINTER(C.c_size_t)]),
    "sbio_server_destroy": (C.c_int, [_vp]),
    "sbio_measure_peaks": (C.c_int, [C.c_int32, C.POINTER(sbio_peaks)]),
    "sbio_geom_set_far_method": (C.c_int, [_vp, C.c_int32, C.c_double, C.c_int32]),
    "sbio_geom_tree_phase_times": (C.c_int, [_vp, _vp]),
    "sbio_geom_tree_info": (C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "sbio_geom_near_work": (C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "sbio_apply_self_noalloc": (C.c_int, [C.POINTER(sbio_spheroid), C.c_int32, C.c_int32, C.c_int32, _vp, _vp,
                                          _vp, _vp, _vp]),
}

EXPORTED = []
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    EXPORTED.append(_name)


def _check(code):
    if code != SBIO_OK:
        raise SbioError(code, _lib.sbio_last_error(None).decode())
    return code


def _ptr(t):
    """Raw address of a torch tensor / numpy array / None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(s):
    if s is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ---- same-name thin wrappers -------------------------------------------------

def sbio_version() -> str:
    return _lib.sbio_version().decode()


def sbio_last_error() -> str:
    return _lib.sbio_last_error(None).decode()


def sbio_launch_count() -> int:
    return int(_lib.sbio_launch_count())


def sbio_ctx_create(device: int = 0, mem_budget_bytes: int = 0):
    h = _vp()
    _check(_lib.sbio_ctx_create(device, mem_budget_bytes, C.byref(h)))
    return h


def sbio_ctx_destroy(ctx):
    _check(_lib.sbio_ctx_destroy(ctx))


def sbio_ctx_mem_used(ctx) -> int:
    b = C.c_size_t()
    _check(_lib.sbio_ctx_mem_used(ctx, C.byref(b)))
    return int(b.value)


def make_spheroids(kind, A, Cax, center, quat):
    M = len(kind)
    arr = (sbio_spheroid * M)()
    for i in range(M):
        arr[i].kind = int(kind[i])
        arr[i].A = float(A[i])
        arr[i].C = float(Cax[i])
        for k in range(3):
            arr[i].center[k] = float(center[i][k])
        for k in range(4):
            arr[i].quat[k] = float(quat[i][k])
    return arr


def sbio_geom_create(ctx, spheroids, p, n_phi=0, near_factor=1.0, precision=SBIO_FP64, stream=None,
                     far_upsample=1):
    opts = sbio_options(p, n_phi, near_factor, far_upsample, precision)
    h = _vp()
    _check(_lib.sbio_geom_create(ctx, spheroids, len(spheroids), C.byref(opts), _stream(stream), C.byref(h)))
    return h


def sbio_geom_destroy(g):
    _check(_lib.sbio_geom_destroy(g))


def sbio_geom_info(g):
    nt, nn, nf, b = C.c_int64(), C.c_int64(), C.c_int64(), C.c_size_t()
    _check(_lib.sbio_geom_info(g, C.byref(nt), C.byref(nn), C.byref(nf), C.byref(b)))
    return {"n_targets": nt.value, "n_near_pairs": nn.value, "n_far_pairs": nf.value, "device_bytes": b.value}


def sbio_geom_setup_times(g):
    """(host nodes/multipliers, near sets, device tables + upload) in ms."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(_lib.sbio_geom_setup_times(g, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def sbio_geom_nodes(g):
    n = sbio_geom_info(g)["n_targets"]
    xyz = np.zeros((n, 3))
    nrm = np.zeros((n, 3))
    w = np.zeros(n)
    _check(_lib.sbio_geom_nodes(g, xyz.ctypes.data, nrm.ctypes.data, w.ctypes.data))
    return xyz, nrm, w


def sbio_geom_near_pairs(g):
    n = sbio_geom_info(g)["n_near_pairs"]
    t = np.zeros(n, dtype=np.int32)
    s = np.zeros(n, dtype=np.int32)
    _check(_lib.sbio_geom_near_pairs(g, t.ctypes.data, s.ctypes.data))
    return t, s


def sbio_geom_set_precision(g, precision):
    _check(_lib.sbio_geom_set_precision(g, precision))


def sbio_geom_set_overlap(g, on=True):
    _check(_lib.sbio_geom_set_overlap(g, 1 if on else 0))


def sbio_geom_set_near_cap(g, ctas_per_sm):
    _check(_lib.sbio_geom_set_near_cap(g, ctas_per_sm))


def sbio_geom_set_tree_near_cap(g, ctas_per_sm):
    _check(_lib.sbio_geom_set_tree_near_cap(g, ctas_per_sm))


def sbio_geom_get_tree_near_cap(g):
    a = C.c_int32()
    _check(_lib.sbio_geom_get_tree_near_cap(g, C.byref(a)))
    return a.value


def sbio_geom_get_tuning(g):
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check(_lib.sbio_geom_get_tuning(g, C.byref(a), C.byref(b), C.byref(c)))
    return {"far_tt": a.value, "far_splits": b.value, "near_ctas_per_sm": c.value}


def sbio_geom_set_launch_shape(g, far_tt, far_splits):
    _check(_lib.sbio_geom_set_launch_shape(g, far_tt, far_splits))


def sbio_geom_autotune(g, stream=None):
    """Pick the fastest far-field launch shape; returns (tt, splits, ms)."""
    a, b, c = C.c_int32(), C.c_int32(), C.c_double()
    _check(_lib.sbio_geom_autotune(g, _stream(stream), C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def sbio_geom_enable_timing(g, on=True):
    _check(_lib.sbio_geom_enable_timing(g, 1 if on else 0))


def sbio_geom_phase_times(g):
    """(synth, near, far) milliseconds of the last apply (timing enabled)."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(_lib.sbio_geom_phase_times(g, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def sbio_apply_laplace(g, sigma_tilde, mu_hat, S_out, D_out, stream=None):
    _check(_lib.sbio_apply_laplace(g, _ptr(sigma_tilde), _ptr(mu_hat), _ptr(S_out), _ptr(D_out), _stream(stream)))


def sbio_apply_laplace_parts(g, sigma_tilde, mu_hat, S_out, D_out, parts, stream=None):
    _check(_lib.sbio_apply_laplace_parts(g, _ptr(sigma_tilde), _ptr(mu_hat), _ptr(S_out), _ptr(D_out), parts,
                                         _stream(stream)))


def sbio_apply_laplace_host(g, sigma_tilde, mu_hat, S_out, D_out, stream=None):
    """Host numpy arrays in and out (C-contiguous float64)."""
    for a in (sigma_tilde, mu_hat, S_out, D_out):
        if a is not None:
            assert a.dtype == np.float64 and a.flags.c_contiguous
    _check(_lib.sbio_apply_laplace_host(g, _ptr(sigma_tilde), _ptr(mu_hat), _ptr(S_out), _ptr(D_out),
                                        _stream(stream)))


def sbio_apply_stokes_sl(g, f_tilde, u_out, stream=None):
    _check(_lib.sbio_apply_stokes_sl(g, _ptr(f_tilde), _ptr(u_out), _stream(stream)))


def sbio_apply_laplace_deriv(g, sigma_tilde, mu_hat, Sp_out, Dp_out, stream=None):
    """S'[sigma] and D'[mu] at all nodes (device tensors; either input may be None)."""
    _check(_lib.sbio_apply_laplace_deriv(g, _ptr(sigma_tilde), _ptr(mu_hat), _ptr(Sp_out), _ptr(Dp_out),
                                         _stream(stream)))


def sbio_forward_transform(g, values, coef_out, modified=False, stream=None):
    """Coefficients (device, M x (p+1)^2) of node values (device, N)."""
    _check(_lib.sbio_forward_transform(g, _ptr(values), 1 if modified else 0, _ptr(coef_out), _stream(stream)))


def _info_dict(info):
    return {"iterations": info.iterations, "restarts": info.restarts, "converged": bool(info.converged),
            "rel_residual": info.rel_residual, "ms": info.ms}


def sbio_solve_dirichlet(g, f_nodes, mu_hat_out, completion=SBIO_COMPLETION_ETA_S, tol=1e-10, max_iter=500,
                         restart=50, sigma_tilde_out=None, charges_out=None, stream=None):
    """Completed double-layer Dirichlet solve; returns the solver info dict."""
    info = sbio_solve_info()
    _check(_lib.sbio_solve_dirichlet(g, _ptr(f_nodes), completion, tol, max_iter, restart, _ptr(mu_hat_out),
                                     _ptr(sigma_tilde_out), _ptr(charges_out), C.byref(info), _stream(stream)))
    return _info_dict(info)


def sbio_solve_neumann(g, g_nodes, rho_tilde_out, tol=1e-10, max_iter=500, restart=50, stream=None):
    """Single-layer Neumann solve; returns the solver info dict."""
    info = sbio_solve_info()
    _check(_lib.sbio_solve_neumann(g, _ptr(g_nodes), tol, max_iter, restart, _ptr(rho_tilde_out), C.byref(info),
                                   _stream(stream)))
    return _info_dict(info)


def sbio_targets_create(g, xyz, stream=None):
    """Resident set of points (host float64 array T x 3) of geometry g."""
    xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
    h = _vp()
    _check(_lib.sbio_targets_create(g, _ptr(xyz) if len(xyz) else None, len(xyz), _stream(stream), C.byref(h)))
    return h.value


def sbio_targets_destroy(ts):
    _check(_lib.sbio_targets_destroy(ts))


def sbio_targets_info(ts):
    a, b, c, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_size_t()
    _check(_lib.sbio_targets_info(ts, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
    return {"n_points": a.value, "n_near_pairs": b.value, "n_far_pairs": c.value, "device_bytes": d.value}


def sbio_eval_targets(ts, sigma_tilde, mu_hat, S_out, D_out, stream=None):
    """S and D at the set's points (device tensors; either input may be None)."""
    _check(_lib.sbio_eval_targets(ts, _ptr(sigma_tilde), _ptr(mu_hat), _ptr(S_out), _ptr(D_out), _stream(stream)))


def sbio_apply_laplace_limit(g, sigma_tilde, mu_hat, S_out, D_out, side, stream=None):
    """S and the one-sided limit of D (side +1 exterior, -1 interior, 0 principal value)."""
    _check(_lib.sbio_apply_laplace_limit(g, _ptr(sigma_tilde), _ptr(mu_hat), _ptr(S_out), _ptr(D_out), side,
                                         _stream(stream)))


def sbio_apply_laplace_deriv_limit(g, sigma_tilde, mu_hat, Sp_out, Dp_out, side, stream=None):
    """The one-sided limit of S' (side +1 exterior, -1 interior, 0 principal value) and D'."""
    _check(_lib.sbio_apply_laplace_deriv_limit(g, _ptr(sigma_tilde), _ptr(mu_hat), _ptr(Sp_out), _ptr(Dp_out), side,
                                               _stream(stream)))


def sbio_eval_targets_deriv(ts, dirs, sigma_tilde, mu_hat, Sp_out, Dp_out, stream=None):
    """Directional derivatives of S and D at the set's points along dirs
    (device T x 3); device tensors, either density may be None."""
    _check(_lib.sbio_eval_targets_deriv(ts, _ptr(dirs), _ptr(sigma_tilde), _ptr(mu_hat), _ptr(Sp_out), _ptr(Dp_out),
                                        _stream(stream)))


def sbio_eval_targets_stokes(ts, f_tilde, u_out, p_out=None, stream=None):
    """Stokes velocity (T x 3) and optionally pressure (T) at the set's points."""
    _check(_lib.sbio_eval_targets_stokes(ts, _ptr(f_tilde), _ptr(u_out), _ptr(p_out), _stream(stream)))


def sbio_apply_stokes_dl(g, q_hat, u_out, stream=None):
    """Stokes double layer (principal value) at all nodes; device tensors."""
    _check(_lib.sbio_apply_stokes_dl(g, _ptr(q_hat), _ptr(u_out), _stream(stream)))


def sbio_apply_stokes_dl_limit(g, q_hat, u_out, side, stream=None):
    """Stokes double layer at all nodes, one-sided limit (+1 exterior, -1 interior, 0 principal value)."""
    _check(_lib.sbio_apply_stokes_dl_limit(g, _ptr(q_hat), _ptr(u_out), side, _stream(stream)))


def sbio_eval_targets_stokes_dl(ts, q_hat, u_out, stream=None):
    """Stokes double layer at the set's points; device tensors."""
    _check(_lib.sbio_eval_targets_stokes_dl(ts, _ptr(q_hat), _ptr(u_out), _stream(stream)))


def sbio_apply_stokes_sl_host(g, f_tilde, u_out, stream=None):
    """Host numpy arrays in and out (C-contiguous float64)."""
    for a in (f_tilde, u_out):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _check(_lib.sbio_apply_stokes_sl_host(g, _ptr(f_tilde), _ptr(u_out), _stream(stream)))


def sbio_geom_set_stokes_tuning(g, far_tt, far_splits, near_ctas_per_sm=0):
    _check(_lib.sbio_geom_set_stokes_tuning(g, far_tt, far_splits, near_ctas_per_sm))


def sbio_geom_get_stokes_tuning(g):
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check(_lib.sbio_geom_get_stokes_tuning(g, C.byref(a), C.byref(b), C.byref(c)))
    return {"far_tt": a.value, "far_splits": b.value, "near_ctas_per_sm": c.value}


def sbio_geom_autotune_stokes(g, stream=None):
    """Pick the fastest Stokes far-field shape and near cap; returns (tt, splits, ms)."""
    a, b, c = C.c_int32(), C.c_int32(), C.c_double()
    _check(_lib.sbio_geom_autotune_stokes(g, _stream(stream), C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


SBIO_FAR_DIRECT = 0
SBIO_FAR_TREE = 1


def sbio_geom_set_far_method(g, method, theta=0.5, order=16):
    """Far field by the direct sum (SBIO_FAR_DIRECT) or the particle treecode
    (SBIO_FAR_TREE, mixed S + D applies at the nodes)."""
    _check(_lib.sbio_geom_set_far_method(g, method, theta, order))


def sbio_geom_tree_phase_times(g):
    """(leaf multipoles, translations, direct part, evaluations) in ms of the
    last timed apply."""
    out = (C.c_double * 4)()
    _check(_lib.sbio_geom_tree_phase_times(g, out))
    return tuple(out)


def sbio_geom_tree_info(g):
    a, b, c, d, e = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    _check(_lib.sbio_geom_tree_info(g, C.byref(a), C.byref(b), C.byref(c), C.byref(d), C.byref(e)))
    return {"nodes": a.value, "groups": b.value, "m2p_pairs": c.value, "m2p_source_pairs": d.value,
            "direct_pairs": e.value}


def sbio_geom_tree_order_counts(g, op=0):
    """(target, multipole node) evaluations per apply of operator `op`
    (SBIO_OP_LAPLACE or SBIO_OP_STOKES) at orders 8, 12, 16."""
    a = (C.c_int64 * 3)()
    _check(_lib.sbio_geom_tree_order_counts(g, op, a))
    return {8: a[0], 12: a[1], 16: a[2]}


def sbio_geom_near_work(g):
    """(near pairs, total Miller steps over them) of the S + D near kernel."""
    a, b = C.c_int64(), C.c_int64()
    _check(_lib.sbio_geom_near_work(g, C.byref(a), C.byref(b)))
    return a.value, b.value


def sbio_measure_peaks(device=0):
    """Measured FP32 / f32x2 / MUFU rsqrt / FP64 rates and the far pair's
    register-only rate of one GPU (see include/sbio.h); returns a dict."""
    out = sbio_peaks()
    _check(_lib.sbio_measure_peaks(device, C.byref(out)))
    return {k: getattr(out, k) for k, _ in sbio_peaks._fields_ if k != "reserved"}


def sbio_apply_self_noalloc(spheroids, p, sigma_tilde, mu_hat, S_out, D_out, n_phi=0, stream=None):
    """Self interaction without any device allocation by the library (see
    include/sbio.h): for callers whose device memory is owned by someone else."""
    _check(_lib.sbio_apply_self_noalloc(spheroids, len(spheroids), p, n_phi, _ptr(sigma_tilde), _ptr(mu_hat),
                                        _ptr(S_out), _ptr(D_out), _stream(stream)))


def _ptr_array(ts):
    arr = (_vp * len(ts))()
    for k, t in enumerate(ts):
        arr[k] = _ptr(t)
    return arr


def sbio_batch_create(ctx, geoms):
    hs = (_vp * len(geoms))(*[g.h if hasattr(g, "h") else g for g in geoms])
    h = _vp()
    _check(_lib.sbio_batch_create(ctx, hs, len(geoms), C.byref(h)))
    return h


def sbio_batch_destroy(b):
    _check(_lib.sbio_batch_destroy(b))


def sbio_batch_info(b):
    a, c, d, e = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int32()
    _check(_lib.sbio_batch_info(b, C.byref(a), C.byref(c), C.byref(d), C.byref(e)))
    return {"n_items": a.value, "far_pairs": c.value, "far_tt": d.value, "grid": e.value}


def sbio_batch_set_far_tt(b, tt):
    _check(_lib.sbio_batch_set_far_tt(b, tt))


def sbio_batch_apply(b, sigmas, mus, S_outs, D_outs, stream=None):
    _check(_lib.sbio_batch_apply(b, _ptr_array(sigmas), _ptr_array(mus), _ptr_array(S_outs), _ptr_array(D_outs),
                                 _stream(stream)))


def sbio_batch_autotune(b, sigmas, mus, S_outs, D_outs, stream=None):
    """Library autotuner of a batch (far targets per thread, near CTA size,
    persistent grid); returns (far_tt, near_block, ctas_per_sm, step_ms)."""
    a, nb, c, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
    _check(_lib.sbio_batch_autotune(b, _ptr_array(sigmas), _ptr_array(mus), _ptr_array(S_outs), _ptr_array(D_outs),
                                    _stream(stream), C.byref(a), C.byref(nb), C.byref(c), C.byref(ms)))
    return a.value, nb.value, c.value, ms.value


def sbio_server_create(ctx, n_slots, mem_budget_bytes=0):
    h = _vp()
    _check(_lib.sbio_server_create(ctx, n_slots, mem_budget_bytes, C.byref(h)))
    return h


SBIO_REQ_TREE = 1


def sbio_server_submit(srv, op, spheroids, p, coef_host, out_host, n_applies, near_factor=1.0,
                       precision=SBIO_MIXED, n_phi=0, flags=0):
    """coef_host / out_host: C-contiguous float64 numpy arrays kept alive by
    the caller until sbio_server_wait returns for the ticket.  flags:
    SBIO_REQ_TREE for the treecode far field (mixed Laplace requests)."""
    req = sbio_request(op, n_applies, C.cast(spheroids, C.c_void_p), len(spheroids), flags,
                       sbio_options(p, n_phi, near_factor, 1, precision), coef_host.ctypes.data,
                       out_host.ctypes.data)
    t = C.c_int64()
    _check(_lib.sbio_server_submit(srv, C.byref(req), C.byref(t)))
    return t.value


def sbio_server_wait(srv, ticket, timeout_s=600.0):
    """Returns (status, latency_ms, service_ms)."""
    st, lat, svc = C.c_int32(), C.c_double(), C.c_double()
    _check(_lib.sbio_server_wait(srv, ticket, timeout_s, C.byref(st), C.byref(lat), C.byref(svc)))
    return st.value, lat.value, svc.value


def sbio_server_stats(srv):
    a, b, c, d, e = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int32(), C.c_size_t()
    _check(_lib.sbio_server_stats(srv, C.byref(a), C.byref(b), C.byref(c), C.byref(d), C.byref(e)))
    return {"completed": a.value, "applies": b.value, "running": c.value, "queued": d.value, "reserved": e.value}


def sbio_server_destroy(srv):
    _check(_lib.sbio_server_destroy(srv))


# ---- convenience object ------------------------------------------------------

class Geometry:
    """Resident geometry of one suspension (owns its library handle)."""

    def __init__(self, ctx, susp, p=None, near_factor=1.0, precision=SBIO_FP64, n_phi=0, stream=None):
        self.ctx = ctx
        self.p = susp.p if p is None else p
        sph = make_spheroids(susp.kind, susp.A, susp.C, susp.center, susp.quat)
        self.h = sbio_geom_create(ctx, sph, self.p, n_phi, near_factor, precision, stream)
        self.M = len(sph)
        info = sbio_geom_info(self.h)
        self.N = info["n_targets"]
        self.n_near = info["n_near_pairs"]
        self.n_far = info["n_far_pairs"]
        self.device_bytes = info["device_bytes"]

    def close(self):
        if self.h:
            sbio_geom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TargetSet:
    """Resident points of a geometry for particle-to-target evaluation."""

    def __init__(self, geom, xyz, stream=None):
        self.geom = geom
        self.h = sbio_targets_create(geom.h, xyz, stream)
        info = sbio_targets_info(self.h)
        self.T = info["n_points"]
        self.n_near = info["n_near_pairs"]
        self.n_far = info["n_far_pairs"]

    def close(self):
        if self.h:
            sbio_targets_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
