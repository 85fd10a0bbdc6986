"""ctypes binding of the plain FP64 oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark. The product path never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def compile_library(src: str, out: str) -> str:
    """gcc -O2 without fused multiply-add contraction, src -> shared library out."""
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", src,
                           "-o", tmp, "-lm", "-lpthread"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, no fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_library(_SRC, _LIB)
    return _LIB


def load(path: str):
    """ctypes handle of an oracle library at path, with every export's argument types."""
    L = C.CDLL(path)
    L.oracle_n_ao.argtypes = [C.c_int, _ip]
    L.oracle_ao_eval.argtypes = [C.c_int, _ip, _ip, _ip, _dp, _dp, _dp, C.c_int, _dp, _dp]
    L.oracle_mo_eval.argtypes = [C.c_int, _ip, _ip, _ip, _dp, _dp, _dp, C.c_int, _dp, C.c_int, _dp, _dp]
    L.oracle_det.argtypes = [C.c_int, _dp, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.oracle_inverse.argtypes = [C.c_int, _dp, _dp]
    L.oracle_evaluate.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp,
                                  C.c_int, _ip, _ip, _ip, _dp, _dp, C.c_int, _dp,
                                  C.c_int64, C.c_int, _up, _up, _dp, C.c_int64, _dp, C.c_int, C.c_int,
                                  _dp, _ip, _dp, _dp, _dp, _dp]
    L.oracle_spin_dets.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _ip, _ip, _ip, _dp, _dp, _dp,
                                   C.c_int, _dp, C.c_int64, C.c_int, _up, C.c_int64, _dp, C.c_int,
                                   _dp, _ip, _dp]
    L.oracle_potential.argtypes = [C.c_int, _dp, C.c_int, _dp, _dp]
    L.oracle_potential.restype = C.c_double
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(_LIB)
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _basis(wl):
    return (len(wl.shell_l), _i32(wl.shell_l), _i32(wl.shell_center), _i32(wl.shell_nprim),
            _f64(wl.alpha), _f64(wl.coef), _f64(wl.nuc_xyz))


def _mo_colmajor(wl):
    # n_ao x n_mo column-major == the transpose stored row-major
    return _f64(np.asarray(wl.mo_coef).T)


def ao_eval(wl, pts):
    pts = _f64(pts).reshape(-1, 3)
    n_ao = wl.n_ao
    out = np.empty((pts.shape[0], 5, n_ao))
    rc = lib().oracle_ao_eval(*_basis(wl), pts.shape[0], pts, out)
    assert rc == 0, rc
    return out


def mo_eval(wl, pts, mo_coef=None):
    pts = _f64(pts).reshape(-1, 3)
    mo = wl.mo_coef if mo_coef is None else mo_coef
    n_mo = mo.shape[1]
    out = np.empty((pts.shape[0], 5, n_mo))
    rc = lib().oracle_mo_eval(*_basis(wl), n_mo, _f64(np.asarray(mo).T), pts.shape[0], pts, out)
    assert rc == 0, rc
    return out


def det(a):
    a = _f64(a)
    n = a.shape[0]
    la, sg = C.c_double(), C.c_int()
    rc = lib().oracle_det(n, a, C.byref(la), C.byref(sg))
    assert rc == 0
    return la.value, sg.value


def inverse(a):
    a = _f64(a)
    out = np.empty_like(a)
    rc = lib().oracle_inverse(a.shape[0], a, out)
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    return out


def evaluate(wl, R=None, mode=0, n_threads=None, mo_coef=None, det_up=None, det_dn=None, ci=None):
    """Oracle log|Psi|, sign, grad Psi/Psi, Lap_i Psi/Psi, E_L and kappa."""
    R = _f64(wl.R if R is None else R)
    n_walk = R.shape[0]
    ne = wl.n_up + wl.n_dn
    mo = wl.mo_coef if mo_coef is None else mo_coef
    du = np.ascontiguousarray(wl.det_up if det_up is None else det_up, dtype=np.uint64)
    dd = np.ascontiguousarray(wl.det_dn if det_dn is None else det_dn, dtype=np.uint64)
    cc = _f64(wl.ci_coef if ci is None else ci)
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    out = dict(log_abs_psi=np.empty(n_walk), sign=np.empty(n_walk, np.int32),
               grad=np.empty((n_walk, ne, 3)), lap=np.empty((n_walk, ne)),
               e_local=np.empty(n_walk), kappa=np.empty(n_walk))
    if n_walk == 0:
        return out
    rc = lib().oracle_evaluate(wl.n_up, wl.n_dn, len(wl.Z), _f64(wl.Z), _f64(wl.nuc_xyz),
                               *_basis(wl)[:6], mo.shape[1], _f64(np.asarray(mo).T),
                               cc.shape[0], du.shape[1], du, dd, cc, n_walk, R, mode, int(n_threads),
                               out["log_abs_psi"], out["sign"], out["grad"], out["lap"],
                               out["e_local"], out["kappa"])
    if rc != 0:
        raise ValueError("oracle_evaluate failed: %d" % rc)
    return out


def potential(r, Z=(), X=()):
    """V = -sum_iA Z_A / |r_i - X_A| + sum_{i<j} 1 / |r_i - r_j| + sum_{A<B} Z_A Z_B / |X_A - X_B|."""
    r = _f64(r).reshape(-1, 3)
    Z = _f64(Z).reshape(-1)
    X = _f64(X).reshape(-1, 3)
    assert X.shape[0] == Z.shape[0]
    return lib().oracle_potential(r.shape[0], r, Z.shape[0], Z if Z.size else np.zeros(1),
                                  X if X.size else np.zeros((1, 3)))


def spin_dets(wl, spin, dets, R=None, mode=0, mo_coef=None):
    """log|D|, sign and (d_{i mu} D)/D of the given spin determinants at each walker."""
    R = _f64(wl.R if R is None else R)
    n_walk = R.shape[0]
    ne = wl.n_up + wl.n_dn
    n = wl.n_up if spin == 0 else wl.n_dn
    e0 = 0 if spin == 0 else wl.n_up
    dets = np.ascontiguousarray(dets, dtype=np.uint64)
    nd = dets.shape[0]
    mo = wl.mo_coef if mo_coef is None else mo_coef
    out_log = np.empty((n_walk, nd))
    out_sign = np.empty((n_walk, nd), np.int32)
    out_dd = np.empty((n_walk, nd, n, 4))
    rc = lib().oracle_spin_dets(ne, e0, n, *_basis(wl)[:6], _f64(wl.nuc_xyz), mo.shape[1],
                                _f64(np.asarray(mo).T), nd, dets.shape[1], dets, n_walk, R, mode,
                                out_log, out_sign, out_dd)
    assert rc == 0, rc
    return out_log, out_sign, out_dd
