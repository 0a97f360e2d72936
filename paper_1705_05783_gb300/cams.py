"""Thin ctypes binding of include/cams.h (argument marshalling only).

Each function has the name of the C entry point it calls.  Arrays are
passed as numpy float64/int32 arrays (memspace CAMS_HOST) or as CUDA torch
tensors (memspace CAMS_DEVICE); nothing here computes any part of the
method.  Importing this module loads the in-tree libcams.so and fails loudly
when it is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcams.so")

CAMS_OK, CAMS_EINVAL, CAMS_ENOMEM, CAMS_ECUDA = 0, -1, -2, -3
CAMS_ENOCONV, CAMS_ESINGULAR, CAMS_ETIMEOUT, CAMS_ENAN = -4, -5, -6, -7
CAMS_HOST, CAMS_DEVICE = 0, 1
CAMS_PREC_FP64, CAMS_PREC_MIXED = 0, 1
CAMS_Q_TRANS, CAMS_Q_MATRIX, CAMS_Q_RHS, CAMS_Q_EPS, CAMS_Q_PRESSURE = 1, 2, 3, 4, 5
CAMS_Q_PROLONG, CAMS_Q_PROLONG_J, CAMS_Q_COARSE, CAMS_Q_ILU_DIAG, CAMS_Q_RESIDUAL = 6, 7, 8, 9, 10
CAMS_Q_SIZES, CAMS_Q_PROFILE, CAMS_Q_LAUNCHES, CAMS_Q_SURR_RATIO = 11, 12, 13, 14
CAMS_Q_MATRIX_UPPER = 15
CAMS_Q_COARSE_FACTOR, CAMS_Q_COARSE_ORDER = 16, 17
PROF_CLASSES = ("assemble", "basis_op", "adapt", "basis", "galerkin", "coarse_factor",
                "ilu_factor", "residual", "restrict", "coarse_solve", "prolong", "ilu_fwd",
                "ilu_bwd", "ilu_resid", "update", "ilu_apply", "coarse_inv")

EXPORTS = ("cams_setup", "cams_set_permeability", "cams_profile", "cams_selftest_wait",
           "cams_set_stream", "cams_set_schedule", "cams_get_schedule",
           "cams_assemble", "cams_update_basis", "cams_iterate", "cams_solve",
           "cams_ensemble_solve", "cams_set_surrogate", "cams_surrogate_data",
           "cams_net_conv_forward", "cams_net_conv_backward", "cams_net_mse", "cams_net_energy",
           "cams_net_adam", "cams_net_tc_work_bytes", "cams_net_conv_forward_tc",
           "cams_net_forward_tc",
           "cams_get",
           "cams_get_int", "cams_last_error", "cams_destroy", "cams_residual_norm_noalloc")


class CamsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cams error {code}: {msg}")
        self.code = code


class cams_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double)]


class cams_fluid(C.Structure):
    _fields_ = [("law", C.c_int), ("c_or_eta", C.c_double), ("rho0", C.c_double),
                ("mu", C.c_double), ("phi", C.c_double)]


class cams_bc(C.Structure):
    _fields_ = [("dirichlet", C.c_int), ("p_west", C.c_double), ("p_east", C.c_double),
                ("n_src", C.c_int), ("src_cell", C.c_void_p), ("src_rate", C.c_void_p),
                ("n_fix", C.c_int), ("fix_cell", C.c_void_p), ("fix_value", C.c_void_p)]


class cams_options(C.Structure):
    _fields_ = [("coarse", C.c_int * 3), ("basis", C.c_int), ("restriction", C.c_int),
                ("n_pre", C.c_int), ("n_post", C.c_int), ("lin_rtol", C.c_double),
                ("nl_tol", C.c_double), ("tol_abs", C.c_int), ("adapt_theta", C.c_double),
                ("max_newton", C.c_int), ("max_cams", C.c_int), ("memspace", C.c_int),
                ("precision", C.c_int), ("cf", C.c_int), ("jacobian", C.c_int)]


class cams_stats(C.Structure):
    _fields_ = [("newton_its", C.c_int), ("cams_its", C.c_int), ("basis_rebuilt", C.c_int),
                ("converged", C.c_int), ("cams_per_newton", C.c_int * 64),
                ("eps_hist", C.c_double * 65), ("res_final", C.c_double),
                ("t_assemble", C.c_double), ("t_precond", C.c_double),
                ("t_iterate", C.c_double), ("t_total", C.c_double)]


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libcams.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "cams_setup": (C.c_int, [C.POINTER(cams_grid), C.POINTER(cams_fluid),
                                 C.POINTER(cams_options), P, P, P, C.POINTER(P)]),
        "cams_set_stream": (C.c_int, [P, P]),
        "cams_set_schedule": (C.c_int, [P, C.c_int, C.c_int]),
        "cams_get_schedule": (C.c_int, [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "cams_set_permeability": (C.c_int, [P, P, P, P]),
        "cams_profile": (C.c_int, [P, C.c_int]),
        "cams_selftest_wait": (C.c_int, [P]),
        "cams_assemble": (C.c_int, [P, P, P, C.c_double, C.POINTER(cams_bc),
                                    C.POINTER(C.c_double)]),
        "cams_update_basis": (C.c_int, [P, C.c_int, C.POINTER(C.c_int)]),
        "cams_iterate": (C.c_int, [P, C.c_int, P]),
        "cams_solve": (C.c_int, [P, P, C.c_double, C.POINTER(cams_bc), P,
                                 C.POINTER(cams_stats)]),
        "cams_ensemble_solve": (C.c_int, [C.c_int, P, P, P, P, P, P, P, C.c_int]),
        "cams_set_surrogate": (C.c_int, [P, P, C.c_double]),
        "cams_surrogate_data": (C.c_int, [P, C.c_int, P, P, P, C.POINTER(C.c_int)]),
        "cams_net_conv_forward": (C.c_int, [C.c_int] * 4 + [P, P, P, C.c_int, P, P]),
        "cams_net_conv_backward": (C.c_int, [C.c_int] * 4 + [P] * 7 + [P]),
        "cams_net_mse": (C.c_int, [C.c_longlong, P, P, P, C.c_double, P, P, P, P]),
        "cams_net_energy": (C.c_int, [C.c_int] * 4 + [P] * 4 + [C.c_double, P, P, P, P]),
        "cams_net_adam": (C.c_int, [C.c_longlong, P, P, P, P, C.c_float, C.c_float, C.c_float,
                                    C.c_float, C.c_int, P]),
        "cams_net_tc_work_bytes": (C.c_longlong, [C.c_int, C.c_int]),
        "cams_net_conv_forward_tc": (C.c_int, [C.c_int] * 4 + [P, P, P, C.c_int, P, P, C.c_longlong, P]),
        "cams_net_forward_tc": (C.c_int, [C.c_int, C.c_int, P, P, P, P, C.c_longlong, P]),
        "cams_get": (C.c_int, [P, C.c_int, P]),
        "cams_get_int": (C.c_int, [P, C.c_int, P]),
        "cams_last_error": (C.c_char_p, [P]),
        "cams_destroy": (None, [P]),
        "cams_residual_norm_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, P, P, P, P, P, P, P,
                                                 C.POINTER(C.c_double), P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


def _ptr(a):
    """Address of a numpy array (host) or a CUDA tensor (device)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _check(code, h=None):
    if code != CAMS_OK:
        raise CamsError(code, _lib.cams_last_error(h).decode())


def make_bc(dirichlet=True, p_west=1.0, p_east=0.0, src_cell=None, src_rate=None,
            fix_cell=None, fix_value=None):
    """cams_bc plus the arrays it points to (kept alive by the returned tuple)."""
    keep = []
    n = 0 if src_cell is None else len(src_cell)
    nf = 0 if fix_cell is None else len(fix_cell)
    bc = cams_bc(int(bool(dirichlet)), float(p_west), float(p_east), n, None, None, nf, None, None)
    if n:
        if isinstance(src_cell, np.ndarray):
            src_cell = np.ascontiguousarray(src_cell, dtype=np.int32)
            src_rate = np.ascontiguousarray(src_rate, dtype=np.float64)
        keep += [src_cell, src_rate]
        bc.src_cell = _ptr(src_cell)
        bc.src_rate = _ptr(src_rate)
    if nf:
        if isinstance(fix_cell, np.ndarray):
            fix_cell = np.ascontiguousarray(fix_cell, dtype=np.int32)
            fix_value = np.ascontiguousarray(fix_value, dtype=np.float64)
        keep += [fix_cell, fix_value]
        bc.fix_cell = _ptr(fix_cell)
        bc.fix_value = _ptr(fix_value)
    return bc, keep


def make_options(coarse, basis=4, restriction=0, n_pre=0, n_post=1, lin_rtol=0.1,
                 nl_tol=1e-6, tol_abs=False, adapt_theta=0.1, max_newton=50, max_cams=200,
                 memspace=CAMS_HOST, precision=CAMS_PREC_FP64, cf=False, jacobian=0):
    """A cams_options (fields as documented in cams.h); cf turns the
    correction functions on, jacobian = 1 selects the full-Jacobian Newton
    step."""
    o = cams_options()
    o.coarse[:] = [int(v) for v in coarse]
    o.basis, o.restriction, o.n_pre, o.n_post = int(basis), int(restriction), int(n_pre), int(n_post)
    o.lin_rtol, o.nl_tol, o.tol_abs = float(lin_rtol), float(nl_tol), int(bool(tol_abs))
    o.adapt_theta, o.max_newton, o.max_cams = float(adapt_theta), int(max_newton), int(max_cams)
    o.memspace = int(memspace)
    o.precision = int(precision)
    o.cf = int(bool(cf))
    o.jacobian = int(jacobian)
    return o


def cams_setup(grid: cams_grid, fluid: cams_fluid, opt: cams_options, kx, ky=None, kz=None):
    h = C.c_void_p()
    code = _lib.cams_setup(C.byref(grid), C.byref(fluid), C.byref(opt), _ptr(kx), _ptr(ky),
                           _ptr(kz), C.byref(h))
    _check(code, None)
    return h


def cams_set_permeability(h, kx, ky=None, kz=None):
    _check(_lib.cams_set_permeability(h, _ptr(kx), _ptr(ky), _ptr(kz)), h)


def cams_profile(h, enable=True):
    _check(_lib.cams_profile(h, int(bool(enable))), h)


def profile_table(h):
    """{class name: (launch groups, total ms, kernels)} from CAMS_Q_PROFILE."""
    a = np.zeros(3 * len(PROF_CLASSES))
    _check(_lib.cams_get(h, CAMS_Q_PROFILE, a.ctypes.data), h)
    return {n: (int(a[3 * k]), float(a[3 * k + 1]), int(a[3 * k + 2]))
            for k, n in enumerate(PROF_CLASSES)}


def cams_selftest_wait(h):
    """Returns the status code (CAMS_ETIMEOUT expected) without raising."""
    return _lib.cams_selftest_wait(h)


def launches(h):
    a = np.zeros(1)
    _check(_lib.cams_get(h, CAMS_Q_LAUNCHES, a.ctypes.data), h)
    return int(a[0])


def cams_set_stream(h, stream_ptr: int):
    _check(_lib.cams_set_stream(h, C.c_void_p(stream_ptr)), h)


def cams_set_schedule(h, ilu_cta=-1, coarse_cluster=-1):
    _check(_lib.cams_set_schedule(h, int(ilu_cta), int(coarse_cluster)), h)


def cams_get_schedule(h):
    """(ilu_cta, coarse_cluster) of the handle."""
    a, b = C.c_int(0), C.c_int(0)
    _check(_lib.cams_get_schedule(h, C.byref(a), C.byref(b)), h)
    return a.value, b.value


def cams_assemble(h, p_nu, p_n, dt, bc):
    e = C.c_double()
    _check(_lib.cams_assemble(h, _ptr(p_nu), _ptr(p_n), float(dt), C.byref(bc), C.byref(e)), h)
    return e.value


def cams_update_basis(h, force=False):
    n = C.c_int()
    _check(_lib.cams_update_basis(h, int(bool(force)), C.byref(n)), h)
    return n.value


def cams_iterate(h, n):
    out = np.zeros(n + 1)
    _check(_lib.cams_iterate(h, int(n), out.ctypes.data), h)
    return out


def cams_solve(h, p_n, dt, bc, p_inout, allow_noconv=False):
    st = cams_stats()
    code = _lib.cams_solve(h, _ptr(p_n), float(dt), C.byref(bc), _ptr(p_inout), C.byref(st))
    if not (allow_noconv and code == CAMS_ENOCONV):
        _check(code, h)
    return st


def cams_ensemble_solve(hs, p_ns, dts, bcs, p_inouts, n_workers=0):
    """cams_ensemble_solve over lists of equal length.  Returns
    (status list, cams_stats list); raises on a bad-argument error."""
    n = len(hs)
    H = (C.c_void_p * n)(*[h.value for h in hs])
    PN = (C.c_void_p * n)(*[_ptr(a) for a in p_ns])
    PI = (C.c_void_p * n)(*[_ptr(a) for a in p_inouts])
    DT = (C.c_double * n)(*[float(d) for d in dts])
    BC = (C.c_void_p * n)(*[C.addressof(b) for b in bcs])
    ST = (cams_stats * n)()
    SS = (C.c_int * n)()
    code = _lib.cams_ensemble_solve(n, H, PN, DT, BC, PI, ST, SS, int(n_workers))
    if code == CAMS_EINVAL and all(s == CAMS_OK for s in SS):
        raise CamsError(code, _lib.cams_last_error(None).decode())
    return list(SS), list(ST)


CAMS_NET_IN, CAMS_NET_HID, CAMS_NET_OUT, CAMS_NET_PARAMS = 12, 32, 8, 72680


def cams_set_surrogate(h, params, gate_tol):
    """params: float32 host array of CAMS_NET_PARAMS values (None with
    gate_tol <= 0 disables the surrogate)."""
    if params is not None:
        params = np.ascontiguousarray(params, dtype=np.float32)
        if params.size != CAMS_NET_PARAMS:
            raise ValueError("wrong number of surrogate parameters")
    _check(_lib.cams_set_surrogate(h, _ptr(params), float(gate_tol)), h)


def cams_surrogate_data(h, max_patches, x=None, target=None, mask=None):
    """Writes up to max_patches training patches into the device tensors;
    returns the number written."""
    n = C.c_int(0)
    _check(_lib.cams_surrogate_data(h, int(max_patches), _ptr(x), _ptr(target), _ptr(mask),
                                    C.byref(n)), h)
    return n.value


def _stream(stream):
    return None if stream is None else int(stream)


def cams_net_conv_forward(B, S, ci, co, x, w, b, relu, y, stream=None):
    _check(_lib.cams_net_conv_forward(B, S, ci, co, _ptr(x), _ptr(w), _ptr(b), int(relu),
                                      _ptr(y), _stream(stream)))


def cams_net_conv_backward(B, S, ci, co, x, w, gy, xact, gx, gw, gb, stream=None):
    _check(_lib.cams_net_conv_backward(B, S, ci, co, _ptr(x), _ptr(w), _ptr(gy), _ptr(xact),
                                       _ptr(gx), _ptr(gw), _ptr(gb), _stream(stream)))


def cams_net_mse(n, pred, target, mask, count, grad, loss, scratch, stream=None):
    _check(_lib.cams_net_mse(int(n), _ptr(pred), _ptr(target), _ptr(mask), float(count),
                             _ptr(grad), _ptr(loss), _ptr(scratch), _stream(stream)))


def cams_net_energy(B, S, C_, cx, pred, target, mask, x, count, grad, loss, scratch, stream=None):
    _check(_lib.cams_net_energy(int(B), int(S), int(C_), int(cx), _ptr(pred), _ptr(target),
                                _ptr(mask), _ptr(x), float(count), _ptr(grad), _ptr(loss),
                                _ptr(scratch), _stream(stream)))


def cams_net_adam(n, p, g, m, v, lr, beta1, beta2, eps, step, stream=None):
    _check(_lib.cams_net_adam(int(n), _ptr(p), _ptr(g), _ptr(m), _ptr(v), float(lr),
                              float(beta1), float(beta2), float(eps), int(step), _stream(stream)))


def cams_get(h, what, dst):
    _check(_lib.cams_get(h, int(what), _ptr(dst)), h)
    return dst


def cams_get_int(h, what, dst):
    _check(_lib.cams_get_int(h, int(what), _ptr(dst)), h)
    return dst


def cams_last_error(h=None) -> str:
    return _lib.cams_last_error(h).decode()


def cams_residual_norm_noalloc(nx, ny, nz, diag, ax, ay, az, f, p, r=None, stream_ptr=0,
                               want_norm=True):
    """||f - A p||_2 (and r, if given) with no device allocation; device
    tensors in, Python float out (None when want_norm is false, which passes
    a null norm_out).  Returns (status, norm)."""
    out = C.c_double(0.0)
    code = _lib.cams_residual_norm_noalloc(int(nx), int(ny), int(nz), _ptr(diag), _ptr(ax),
                                           _ptr(ay), _ptr(az), _ptr(f), _ptr(p), _ptr(r),
                                           C.byref(out) if want_norm else None,
                                           C.c_void_p(stream_ptr))
    return code, (out.value if want_norm else None)


def cams_net_tc_work_bytes(B, S):
    """Bytes of device workspace the tensor-core network calls need."""
    return int(_lib.cams_net_tc_work_bytes(int(B), int(S)))


def cams_net_conv_forward_tc(B, S, ci, co, x, w, bias, relu, y, work, work_bytes, stream_ptr=0):
    """One layer on the tensor cores (FP32 in and out, BF16 operands);
    returns the status code."""
    return _lib.cams_net_conv_forward_tc(int(B), int(S), int(ci), int(co), _ptr(x), _ptr(w),
                                         _ptr(bias), int(relu), _ptr(y), _ptr(work),
                                         int(work_bytes), C.c_void_p(stream_ptr))


def cams_net_forward_tc(B, S, x, params, y, work, work_bytes, stream_ptr=0):
    """The whole network on the tensor cores; returns the status code."""
    return _lib.cams_net_forward_tc(int(B), int(S), _ptr(x), _ptr(params), _ptr(y), _ptr(work),
                                    int(work_bytes), C.c_void_p(stream_ptr))


def cams_destroy(h):
    _lib.cams_destroy(h)
