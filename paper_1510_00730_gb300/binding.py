"""Thin ctypes binding of libmdet.so: argument marshalling only.

Names follow the C ABI (include/mdet.h). Device buffers are torch CUDA
tensors; torch provides memory and the current stream, every step of the
evaluation runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

PRECISION_FP64 = 0
PRECISION_MIXED = 1
NO_DEVICE = -1
WS_REF_SINGULAR = 0x1
WS_REF_ILLCOND = 0x2
WS_PSI_ZERO = 0x4
WS_NONFINITE = 0x8
WS_FALLBACK = 0x10
WS_ESCALATED = 0x20
MAX_EXC = 4

_lib = None


class MdetError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


class _Tuning(C.Structure):
    _fields_ = [("spmm_chunk", C.c_int32), ("mo_ec", C.c_int32), ("walker_chunks", C.c_int32),
                ("best_ms", C.c_float), ("trials", C.c_int32), ("spmm_blocks", C.c_int32), ("mo_impl", C.c_int32),
                ("contract_impl", C.c_int32)]


class _Stats(C.Structure):
    _fields_ = [("n_up", C.c_int32), ("n_dn", C.c_int32), ("n_ao", C.c_int32), ("n_mo", C.c_int32),
                ("n_int", C.c_int32), ("n_det", C.c_int64), ("n_det_up", C.c_int32), ("n_det_dn", C.c_int32),
                ("max_degree", C.c_int32 * 2), ("degree_hist", (C.c_int64 * (MAX_EXC + 1)) * 2),
                ("precision", C.c_int32), ("device", C.c_int32)]


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libmdet.so (building it first if allowed). Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError("libmdet.so is not built (run __graft_entry__.build())")
        _build.build()
    L = C.CDLL(_build.LIB)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    L.mdet_create.argtypes = [C.POINTER(vp), i32, i32]
    L.mdet_destroy.argtypes = [vp]
    L.mdet_destroy.restype = None
    L.mdet_status_string.argtypes = [i32]
    L.mdet_status_string.restype = C.c_char_p
    L.mdet_last_error.argtypes = [vp]
    L.mdet_last_error.restype = C.c_char_p
    L.mdet_set_system.argtypes = [vp, i32, i32, i32, vp, vp]
    L.mdet_set_orbitals.argtypes = [vp, i32, vp, vp, vp, vp, vp, i32, vp]
    L.mdet_set_ci_expansion.argtypes = [vp, i64, i32, vp, vp, vp]
    L.mdet_evaluate.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    L.mdet_evaluate_host.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp]
    L.mdet_get_ratios.argtypes = [vp, i64, vp, vp, vp, vp]
    L.mdet_get_stats.argtypes = [vp, C.POINTER(_Stats)]
    L.mdet_get_spin_dets.argtypes = [vp, i32, vp, vp, vp]
    L.mdet_get_ci_matrix.argtypes = [vp, vp, vp, vp]
    L.mdet_omega_sort.argtypes = [i64, i32, vp, vp]
    L.mdet_sm_chain.argtypes = [vp, i64, vp, i64, vp, vp, vp]
    L.mdet_set_ci_expansion_device.argtypes = [vp, i64, i32, vp, vp, vp, vp]
    L.mdet_truncate_norm.argtypes = [i64, i32, vp, vp, vp, C.c_double, C.c_double, vp, vp, vp, vp]
    L.mdet_psi_tilde_noalloc.argtypes = [vp, i64, vp, i64, vp, vp]
    L.mdet_set_profiling.argtypes = [vp, i32]
    L.mdet_set_walker_chunks.argtypes = [vp, i32]
    L.mdet_get_last_launches.argtypes = [vp, vp, vp]
    L.mdet_set_escalation.argtypes = [vp, i32]
    L.mdet_set_fallback.argtypes = [vp, C.c_double, i32]
    L.mdet_get_fallback.argtypes = [vp, vp, vp]
    L.mdet_get_error_estimates.argtypes = [vp, i64, vp, vp]
    L.mdet_selftest_df32.argtypes = [i32, i64, vp, vp, vp, vp]
    L.mdet_selftest_inv_r.argtypes = [i32, i64, vp, vp, vp]
    L.mdet_get_tuning.argtypes = [vp, C.POINTER(_Tuning)]
    L.mdet_set_tuning.argtypes = [vp, C.POINTER(_Tuning)]
    L.mdet_autotune.argtypes = [vp, i64, vp, C.c_double, C.POINTER(_Tuning)]
    pp = C.POINTER(C.c_void_p)
    L.mdet_batch_evaluate.argtypes = [i32, pp, C.POINTER(C.c_int64), pp, pp, pp, pp, pp, pp, pp, i32, vp]
    L.mdet_batch_create.argtypes = [C.POINTER(vp), i32, pp, C.POINTER(C.c_int64), pp, pp, pp, pp, pp, pp, pp, i32]
    L.mdet_batch_launch.argtypes = [vp, vp]
    L.mdet_batch_destroy.argtypes = [vp]
    L.mdet_batch_destroy.restype = None
    L.mdet_get_profile.argtypes = [vp, vp]
    L.mdet_get_timeline.argtypes = [vp, vp, vp]
    L.mdet_measure_fp64_rate.argtypes = [i32, i64, i32, vp, vp, vp]
    for name in ("mdet_create", "mdet_set_system", "mdet_set_orbitals", "mdet_set_ci_expansion", "mdet_evaluate",
                 "mdet_evaluate_host", "mdet_get_ratios", "mdet_get_stats", "mdet_get_spin_dets",
                 "mdet_get_ci_matrix", "mdet_omega_sort", "mdet_truncate_norm", "mdet_sm_chain", "mdet_set_ci_expansion_device", "mdet_set_profiling", "mdet_get_profile",
                 "mdet_psi_tilde_noalloc", "mdet_set_walker_chunks", "mdet_get_last_launches", "mdet_set_escalation", "mdet_selftest_df32", "mdet_selftest_inv_r", "mdet_get_tuning",
                 "mdet_set_tuning", "mdet_autotune", "mdet_batch_evaluate", "mdet_batch_create", "mdet_batch_launch", "mdet_set_fallback", "mdet_get_fallback",
                 "mdet_get_error_estimates", "mdet_measure_fp64_rate", "mdet_get_timeline"):
        getattr(L, name).restype = i32
    # VMC moves and the learned proposal (include/mdet_vmc.h)
    u32p = C.POINTER(C.c_uint32)
    L.mdet_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.mdet_philox4x32_10.restype = None
    L.mdet_vmc_propose_drift.argtypes = [i64, i32, vp, vp, C.c_double, C.c_uint64, C.c_uint64, vp, vp, vp]
    L.mdet_vmc_reverse_drift.argtypes = [i64, i32, vp, vp, vp, C.c_double, vp, vp]
    L.mdet_vmc_accept.argtypes = [i64, i32, C.c_uint64, C.c_uint64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                  vp, vp, vp, vp, vp, vp]
    L.mdet_vmc_r2.argtypes = [i64, i32, vp, vp, vp]
    L.mdet_vmc_select_rows.argtypes = [i64, i32, vp, vp, vp, vp]
    L.mdet_vmc_limit_drift.argtypes = [i64, i32, vp, C.c_double, C.c_double, vp, vp]
    L.mdet_mlp_create.argtypes = [C.POINTER(vp), i32, i32, i32, C.c_uint64, C.c_double, C.c_double, C.c_double,
                                  C.c_double]
    L.mdet_mlp_destroy.argtypes = [vp]
    L.mdet_mlp_destroy.restype = None
    L.mdet_mlp_n_params.argtypes = [vp]
    L.mdet_mlp_n_params.restype = i64
    for n in ("mdet_mlp_get_params", "mdet_mlp_set_params", "mdet_mlp_get_grads"):
        getattr(L, n).argtypes = [vp, vp]
    L.mdet_mlp_forward.argtypes = [vp, i64, vp, vp, vp]
    L.mdet_mlp_backward.argtypes = [vp, i64, vp, vp]
    L.mdet_mlp_zero_grad.argtypes = [vp, vp]
    L.mdet_mlp_adam.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double, i64, vp]
    L.mdet_mlp_nll_grad.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
    L.mdet_vmc_propose_mlp.argtypes = [vp, i64, vp, vp, vp, C.c_uint64, C.c_uint64, vp, vp, vp]
    L.mdet_mlp_esjd_grad.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, C.c_int, C.c_double,
                                     C.c_double, vp, vp, vp, vp]
    L.mdet_vmc_reverse_mlp.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
    L.mdet_gemm_bf16.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, i32, i64, vp]
    for n in ("mdet_gemm_bf16", "mdet_vmc_propose_drift", "mdet_vmc_reverse_drift", "mdet_vmc_accept", "mdet_vmc_r2",
              "mdet_vmc_select_rows", "mdet_vmc_limit_drift",
              "mdet_mlp_create", "mdet_mlp_get_params", "mdet_mlp_set_params", "mdet_mlp_get_grads",
              "mdet_mlp_forward", "mdet_mlp_backward", "mdet_mlp_zero_grad", "mdet_mlp_adam", "mdet_mlp_nll_grad",
              "mdet_vmc_propose_mlp", "mdet_vmc_reverse_mlp", "mdet_mlp_esjd_grad"):
        getattr(L, n).restype = i32
    _lib = L
    return L


def _need(t, name, shape, dtype, device):
    """t must be a contiguous CUDA tensor of exactly this shape and dtype on
    `device`: the kernels read and write that many elements, so any other
    buffer would be an out-of-bounds access. Raises ValueError otherwise."""
    import torch
    ok = (isinstance(t, torch.Tensor) and t.is_cuda and t.device == device and t.dtype == dtype
          and t.is_contiguous() and tuple(t.shape) == tuple(shape))
    if not ok:
        got = ("%s %s on %s%s" % (tuple(t.shape), t.dtype, t.device, "" if t.is_contiguous() else ", strided")
               if isinstance(t, torch.Tensor) else type(t).__name__)
        raise ValueError("%s must be a contiguous %s tensor of shape %s on %s (got %s)" % (name, dtype, tuple(shape),
                                                                                         device, got))
    return t


def _need_np(a, name, shape, dtype):
    """The host counterpart of _need for numpy output arrays."""
    if not (isinstance(a, np.ndarray) and a.dtype == dtype and a.shape == tuple(shape) and a.flags.c_contiguous):
        raise ValueError("%s must be a C-contiguous %s array of shape %s" % (name, np.dtype(dtype), tuple(shape)))
    return a


def _ptr(a) -> int:
    return a.ctypes.data if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def truncate_norm(det_up, det_dn, coef, eps_up, eps_dn):
    """Norm-based truncation (Sec. 3): remove the distinct spin determinants whose
    share of the norm is <= eps_sigma (eps < 0: none) and every product using one.
    Returns (keep [n_det] bool, norm_up [n_det], norm_dn [n_det], counts) with
    counts = dict(products, up, dn, up_all, dn_all)."""
    L = load_library()
    du, dd = _c(det_up, np.uint64), _c(det_dn, np.uint64)
    if du.ndim == 1:
        du, dd = du[:, None], dd[:, None]
    cf = _c(coef, np.float64)
    n = cf.shape[0]
    if du.shape != dd.shape or du.shape[0] != n:
        raise ValueError("det_up, det_dn and coef disagree in length")
    keep = np.empty(n, np.uint8)
    nu, nd = np.empty(n), np.empty(n)
    cnt = np.empty(5, np.int64)
    st = L.mdet_truncate_norm(n, du.shape[1], _ptr(du), _ptr(dd), _ptr(cf), float(eps_up), float(eps_dn),
                              _ptr(keep), _ptr(nu), _ptr(nd), _ptr(cnt))
    if st:
        raise MdetError(st, "mdet_truncate_norm failed")
    return keep.astype(bool), nu, nd, dict(zip(("products", "up", "dn", "up_all", "dn_all"), cnt.tolist()))


def omega_sort(dets) -> np.ndarray:
    """Permutation sorting bit-string determinants [n][n_int] by the key of Eq. 3."""
    L = load_library()
    d = _c(dets, np.uint64)
    if d.ndim == 1:
        d = d[:, None]
    order = np.empty(d.shape[0], np.int64)
    st = L.mdet_omega_sort(d.shape[0], d.shape[1], _ptr(d), _ptr(order))
    if st:
        raise MdetError(st, "mdet_omega_sort failed")
    return order


def selftest_inv_r(x):
    """The Coulomb sums' Newton-refined 1/sqrt against CUDA's FP64 1.0 / sqrt on the
    device (x: CUDA float64)."""
    import torch
    L = load_library()
    y_nr, y_ref = torch.empty_like(x), torch.empty_like(x)
    st = L.mdet_selftest_inv_r(x.device.index or 0, x.numel(), x.data_ptr(), y_nr.data_ptr(), y_ref.data_ptr())
    if st:
        raise MdetError(st, "mdet_selftest_inv_r failed")
    return y_nr, y_ref


def selftest_df32(x):
    """Double-float exp and product against FP64 on the device (x: CUDA float64, <= 0)."""
    import torch
    L = load_library()
    y_df, y_ref, prod = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
    st = L.mdet_selftest_df32(x.device.index or 0, x.numel(), x.data_ptr(), y_df.data_ptr(), y_ref.data_ptr(),
                              prod.data_ptr())
    if st:
        raise MdetError(st, "mdet_selftest_df32 failed")
    return y_df, y_ref, prod


def measure_fp64_rate(device=0, fma_per_thread=1 << 18, reps=10):
    """Measured FP64 FMA throughput of a device: (TFLOP/s, fastest launch in ms, SM MHz during it)."""
    L = load_library()
    tf, ms, mhz = C.c_double(), C.c_double(), C.c_double()
    st = L.mdet_measure_fp64_rate(int(device), int(fma_per_thread), int(reps), C.byref(tf), C.byref(ms),
                                  C.byref(mhz))
    if st:
        raise MdetError(st, "mdet_measure_fp64_rate failed: %s" % L.mdet_status_string(st).decode())
    return tf.value, ms.value, mhz.value


class Context:
    """One expansion resident on one device (or host-only with device=-1)."""

    def __init__(self, device: int = 0, precision: int | str = PRECISION_FP64):
        if isinstance(precision, str):
            precision = {"fp64": PRECISION_FP64, "mixed": PRECISION_MIXED}[precision]
        self._L = load_library()
        h = C.c_void_p()
        st = self._L.mdet_create(C.byref(h), int(device), int(precision))
        if st:
            raise MdetError(st, "mdet_create(device=%d) failed: %s" % (device, self._L.mdet_status_string(st).decode()))
        self._h = h
        self.device = int(device)
        self.precision = int(precision)
        self.n_up = self.n_dn = 0
        self._keep = []

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.mdet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st:
            msg = self._L.mdet_last_error(self._h).decode()
            raise MdetError(st, "%s: %s (%s)" % (what, self._L.mdet_status_string(st).decode(), msg))

    # -- set-up -------------------------------------------------------------
    def set_system(self, n_up, n_dn, Z, nuc_xyz):
        Z = _c(Z, np.float64)
        X = _c(nuc_xyz, np.float64)
        self._check(self._L.mdet_set_system(self._h, int(n_up), int(n_dn), Z.shape[0], _ptr(Z), _ptr(X)),
                    "mdet_set_system")
        self.n_up, self.n_dn = int(n_up), int(n_dn)

    def set_orbitals(self, shell_l, shell_center, shell_nprim, alpha, coef, mo_coef):
        """mo_coef: [n_ao, n_mo] array (column m = MO m)."""
        l_, c_, n_ = _c(shell_l, np.int32), _c(shell_center, np.int32), _c(shell_nprim, np.int32)
        a_, k_ = _c(alpha, np.float64), _c(coef, np.float64)
        mo = np.asarray(mo_coef, dtype=np.float64)
        mo_cm = _c(mo.T, np.float64)  # column-major n_ao x n_mo
        self._check(self._L.mdet_set_orbitals(self._h, l_.shape[0], _ptr(l_), _ptr(c_), _ptr(n_), _ptr(a_), _ptr(k_),
                                              mo.shape[1], _ptr(mo_cm)), "mdet_set_orbitals")

    def set_ci_expansion(self, det_up, det_dn, coef, on_device=False):
        """The CI expansion and its preprocessing; on_device runs the O(N_det)
        steps on the GPU (mdet_set_ci_expansion_device; torch tensors on the
        context's device are used in place, host arrays are copied there)."""
        if on_device:
            import torch
            dev = torch.device("cuda", self.device)
            def words(a):  # 64-bit words in place; torch has no general uint64, so move them as int64 bits
                if isinstance(a, torch.Tensor):
                    return a.to(dev).contiguous()
                return torch.from_numpy(np.ascontiguousarray(a, np.uint64).view(np.int64)).to(dev)

            du, dd = words(det_up), words(det_dn)
            cf = torch.as_tensor(coef, dtype=torch.float64, device=dev).contiguous()
            if du.dim() == 1:
                du, dd = du[:, None].contiguous(), dd[:, None].contiguous()
            self._check(self._L.mdet_set_ci_expansion_device(self._h, cf.shape[0], du.shape[1], du.data_ptr(),
                                                             dd.data_ptr(), cf.data_ptr(), _sp(None, dev)),
                        "mdet_set_ci_expansion_device")
            return
        du, dd, cf = _c(det_up, np.uint64), _c(det_dn, np.uint64), _c(coef, np.float64)
        self._check(self._L.mdet_set_ci_expansion(self._h, cf.shape[0], du.shape[1], _ptr(du), _ptr(dd), _ptr(cf)),
                    "mdet_set_ci_expansion")

    @classmethod
    def from_workload(cls, wl, device=0, precision=PRECISION_FP64, on_device=False):
        ctx = cls(device, precision)
        ctx.set_system(wl.n_up, wl.n_dn, wl.Z, wl.nuc_xyz)
        ctx.set_orbitals(wl.shell_l, wl.shell_center, wl.shell_nprim, wl.alpha, wl.coef, wl.mo_coef)
        ctx.set_ci_expansion(wl.det_up, wl.det_dn, wl.ci_coef, on_device=on_device)
        return ctx

    # -- evaluation ---------------------------------------------------------
    def alloc_outputs(self, n_walk):
        import torch
        dev = torch.device("cuda", self.device)
        N = self.n_up + self.n_dn
        return dict(log_abs_psi=torch.empty(n_walk, dtype=torch.float64, device=dev),
                    sign=torch.empty(n_walk, dtype=torch.int8, device=dev),
                    grad=torch.empty(n_walk, N, 3, dtype=torch.float64, device=dev),
                    lap=torch.empty(n_walk, N, dtype=torch.float64, device=dev),
                    e_local=torch.empty(n_walk, dtype=torch.float64, device=dev),
                    status=torch.empty(n_walk, dtype=torch.int32, device=dev))

    def evaluate(self, R, out=None, stream=None):
        """R: CUDA float64 tensor [n_walk, n_up+n_dn, 3] on this context's device.
        Returns (and fills) a dict of device tensors; asynchronous on `stream`
        (default: torch's current stream)."""
        import torch
        dev = torch.device("cuda", self.device)
        N = self.n_up + self.n_dn
        n_walk = R.shape[0] if isinstance(R, torch.Tensor) and R.dim() == 3 else -1
        _need(R, "R", (n_walk, N, 3), torch.float64, dev)
        if out is None:
            out = self.alloc_outputs(n_walk)
        for k, shape, dt in (("log_abs_psi", (n_walk,), torch.float64), ("sign", (n_walk,), torch.int8),
                             ("grad", (n_walk, N, 3), torch.float64), ("lap", (n_walk, N), torch.float64),
                             ("e_local", (n_walk,), torch.float64), ("status", (n_walk,), torch.int32)):
            _need(out[k], "out['%s']" % k, shape, dt, dev)
        if stream is None:
            stream = torch.cuda.current_stream(R.device)
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._check(self._L.mdet_evaluate(self._h, n_walk, R.data_ptr(), out["log_abs_psi"].data_ptr(),
                                          out["sign"].data_ptr(), out["grad"].data_ptr(), out["lap"].data_ptr(),
                                          out["e_local"].data_ptr(), out["status"].data_ptr(), sp), "mdet_evaluate")
        return out

    def evaluate_host(self, R, out=None):
        """Host-memory evaluation (copies inside the call); returns numpy arrays."""
        R = _c(R, np.float64)
        N = self.n_up + self.n_dn
        if R.ndim != 3 or R.shape[1:] != (N, 3):
            raise ValueError("R must have shape [n_walk, %d, 3]" % N)
        n_walk = R.shape[0]
        if out is None:
            out = dict(log_abs_psi=np.empty(n_walk), sign=np.empty(n_walk, np.int8), grad=np.empty((n_walk, N, 3)),
                       lap=np.empty((n_walk, N)), e_local=np.empty(n_walk), status=np.empty(n_walk, np.uint32))
        for k, shape, dt in (("log_abs_psi", (n_walk,), np.float64), ("sign", (n_walk,), np.int8),
                             ("grad", (n_walk, N, 3), np.float64), ("lap", (n_walk, N), np.float64),
                             ("e_local", (n_walk,), np.float64)):
            _need_np(out[k], "out['%s']" % k, shape, dt)
        if out["status"].shape != (n_walk,) or out["status"].dtype.itemsize != 4:
            raise ValueError("out['status'] must be a 32-bit array of shape (%d,)" % n_walk)
        self._check(self._L.mdet_evaluate_host(self._h, n_walk, _ptr(R), _ptr(out["log_abs_psi"]), _ptr(out["sign"]),
                                               _ptr(out["grad"]), _ptr(out["lap"]), _ptr(out["e_local"]),
                                               _ptr(out["status"])), "mdet_evaluate_host")
        return out

    def ratios(self, n_walk):
        s = self.stats()
        r_up = np.empty((n_walk, s["n_det_up"]))
        r_dn = np.empty((n_walk, s["n_det_dn"]))
        ld0 = np.empty((n_walk, 2))
        sg0 = np.empty((n_walk, 2), np.int8)
        self._check(self._L.mdet_get_ratios(self._h, n_walk, _ptr(r_up), _ptr(r_dn), _ptr(ld0), _ptr(sg0)),
                    "mdet_get_ratios")
        return r_up, r_dn, ld0, sg0

    NOALLOC_SCRATCH_DOUBLES = 4 * 1024 * 1024

    def psi_tilde_noalloc(self, r, ld, psi_tilde, stream=None):
        """Psi~ = r_up . (C r_dn) from walker-minor ratios r (CUDA float64,
        [n_det_up + n_det_dn, ld]) into psi_tilde (CUDA float64, [n_walk]),
        using the library's static scratch instead of any device allocation."""
        import torch
        dev = torch.device("cuda", self.device)
        st = self.stats()
        n_walk = psi_tilde.shape[0] if isinstance(psi_tilde, torch.Tensor) and psi_tilde.dim() == 1 else -1
        _need(psi_tilde, "psi_tilde", (n_walk,), torch.float64, dev)
        _need(r, "r", (st["n_det_up"] + st["n_det_dn"], int(ld)), torch.float64, dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._check(self._L.mdet_psi_tilde_noalloc(self._h, psi_tilde.shape[0], r.data_ptr(), int(ld),
                                                   psi_tilde.data_ptr(), sp), "mdet_psi_tilde_noalloc")

    STAGES = ("orbitals", "reference", "ratios", "zero", "contract", "final")

    def tuning(self):
        t = _Tuning()
        self._check(self._L.mdet_get_tuning(self._h, C.byref(t)), "mdet_get_tuning")
        return dict(spmm_chunk=t.spmm_chunk, mo_ec=t.mo_ec, walker_chunks=t.walker_chunks, best_ms=t.best_ms,
                    trials=t.trials, spmm_blocks=t.spmm_blocks, mo_impl=t.mo_impl,
                    contract_impl=t.contract_impl)

    def set_tuning(self, spmm_chunk=512, mo_ec=None, walker_chunks=0, spmm_blocks=0, mo_impl=None, contract_impl=0):
        """Tile shapes and kernel choices (mdet_set_tuning); mo_ec and mo_impl None keep the
        context's current values."""
        cur = self.tuning()
        if mo_ec is None:
            mo_ec = cur["mo_ec"]
        if mo_impl is None:
            mo_impl = cur["mo_impl"]
        t = _Tuning(spmm_chunk, mo_ec, walker_chunks, 0.0, 0, spmm_blocks, mo_impl, contract_impl)
        self._check(self._L.mdet_set_tuning(self._h, C.byref(t)), "mdet_set_tuning")

    def autotune(self, R, budget_ms=200.0):
        """Pick tile shapes by timing evaluations of the walkers R (CUDA float64)."""
        t = _Tuning()
        self._check(self._L.mdet_autotune(self._h, R.shape[0], R.data_ptr(), float(budget_ms), C.byref(t)),
                    "mdet_autotune")
        return dict(spmm_chunk=t.spmm_chunk, mo_ec=t.mo_ec, walker_chunks=t.walker_chunks, best_ms=t.best_ms,
                    trials=t.trials, spmm_blocks=t.spmm_blocks, mo_impl=t.mo_impl,
                    contract_impl=t.contract_impl)

    ESCALATE_AUTO, ESCALATE_ALWAYS, ESCALATE_NEVER = 0, 1, 2

    def set_escalation(self, mode):
        """Mixed precision: FP64 re-evaluation of flagged walkers before full LU
        (mdet_set_escalation; ESCALATE_AUTO, ESCALATE_ALWAYS or ESCALATE_NEVER)."""
        self._check(self._L.mdet_set_escalation(self._h, int(mode)), "mdet_set_escalation")

    def set_fallback(self, tol, max_walkers=None):
        """Re-evaluate walkers whose estimated table error exceeds tol (tol <= 0: off), at most
        max_walkers per evaluation (None keeps the current cap)."""
        if max_walkers is None:
            max_walkers = self.fallback[1]
        self._check(self._L.mdet_set_fallback(self._h, float(tol), int(max_walkers)), "mdet_set_fallback")

    @property
    def fallback(self):
        """(tolerance, walker cap) of the stability fallback."""
        tol, cap = C.c_double(), C.c_int()
        self._check(self._L.mdet_get_fallback(self._h, C.byref(tol), C.byref(cap)), "mdet_get_fallback")
        return tol.value, cap.value

    def error_estimates(self, n_walk):
        """cond_1 of the references [n_walk, 2] and the table error estimates [n_walk, 2] of the last evaluation."""
        c1 = np.empty((n_walk, 2))
        est = np.empty((n_walk, 2))
        self._check(self._L.mdet_get_error_estimates(self._h, n_walk, _ptr(c1), _ptr(est)), "mdet_get_error_estimates")
        return c1, est

    def set_walker_chunks(self, n_chunks):
        """Mixed precision: pipeline a batch in n_chunks walker chunks (0 = automatic, 1 = none)."""
        self._check(self._L.mdet_set_walker_chunks(self._h, int(n_chunks)), "mdet_set_walker_chunks")

    def _last_launches(self):
        ch, nk = C.c_int32(0), C.c_int32(0)
        self._check(self._L.mdet_get_last_launches(self._h, C.byref(ch), C.byref(nk)), "mdet_get_last_launches")
        return int(ch.value), int(nk.value)

    @property
    def last_chunks(self):
        """Walker chunks of the last evaluation (mdet_get_last_launches; 0 before the first)."""
        return self._last_launches()[0]

    @property
    def last_kernels(self):
        """Kernels the last evaluation launched (mdet_get_last_launches; 0 before the first)."""
        return self._last_launches()[1]

    def set_profiling(self, enable=True):
        """Stage timing: True or 1 events around every stage, 2 the contraction kernels'
        own global-timer stamps (no events in the streams), False or 0 none."""
        mode = enable if isinstance(enable, int) and not isinstance(enable, bool) else int(bool(enable))
        self._check(self._L.mdet_set_profiling(self._h, mode), "mdet_set_profiling")

    def profile(self):
        """Stage durations (ms) of the last profiled evaluation."""
        ms = (C.c_float * len(self.STAGES))()
        self._check(self._L.mdet_get_profile(self._h, ms), "mdet_get_profile")
        return dict(zip(self.STAGES, [float(x) for x in ms]))

    MAX_CHUNKS = 8

    def timeline(self):
        """Start and end (ms after the evaluation's first event) of every stage of every
        walker chunk of the last profiled evaluation, and of the refinement."""
        n = C.c_int32()
        ms = (C.c_float * (2 * self.MAX_CHUNKS * len(self.STAGES) + 3))()
        self._check(self._L.mdet_get_timeline(self._h, C.byref(n), ms), "mdet_get_timeline")
        per = 2 * len(self.STAGES)
        chunks = [{s: (float(ms[k * per + 2 * i]), float(ms[k * per + 2 * i + 1])) for i, s in enumerate(self.STAGES)}
                  for k in range(n.value)]
        tail = ms[self.MAX_CHUNKS * per:]
        return dict(chunks=chunks, refine=(float(tail[0]), float(tail[1])), end=float(tail[2]))

    # -- introspection (host only) -------------------------------------------
    def stats(self):
        s = _Stats()
        self._check(self._L.mdet_get_stats(self._h, C.byref(s)), "mdet_get_stats")
        return dict(n_up=s.n_up, n_dn=s.n_dn, n_ao=s.n_ao, n_mo=s.n_mo, n_int=s.n_int, n_det=s.n_det,
                    n_det_up=s.n_det_up, n_det_dn=s.n_det_dn, max_degree=list(s.max_degree),
                    degree_hist=[list(s.degree_hist[0]), list(s.degree_hist[1])],
                    precision=s.precision, device=s.device)

    def sm_chain(self, n_walk, stream=None):
        """Ratios D_I / D_ref by the paper's sequential Sherman-Morrison chain
        (mdet_sm_chain) on the orbitals of the last evaluation. Returns device
        tensors r [n_det_up + n_det_dn][ld] (walker-minor, ld = n_walk rounded up
        to 256), n_inv [n_walk], n_subst [n_walk]."""
        import torch
        dev = torch.device("cuda", self.device)
        st = self.stats()
        ld = max(256, (n_walk + 255) // 256 * 256)
        r = torch.empty((st["n_det_up"] + st["n_det_dn"], ld), dtype=torch.float64, device=dev)
        n_inv = torch.empty(n_walk, dtype=torch.int32, device=dev)
        n_subst = torch.empty(n_walk, dtype=torch.int32, device=dev)
        self._check(self._L.mdet_sm_chain(self._h, n_walk, r.data_ptr(), ld, n_inv.data_ptr(), n_subst.data_ptr(),
                                          _sp(stream, dev)), "mdet_sm_chain")
        return r, n_inv, n_subst

    def spin_dets(self, spin):
        s = self.stats()
        n = s["n_det_up"] if spin == 0 else s["n_det_dn"]
        dets = np.empty((n, s["n_int"]), np.uint64)
        deg = np.empty(n, np.int32)
        ph = np.empty(n, np.int8)
        self._check(self._L.mdet_get_spin_dets(self._h, int(spin), _ptr(dets), _ptr(deg), _ptr(ph)),
                    "mdet_get_spin_dets")
        return dets, deg, ph

    def ci_matrix(self):
        n = self.stats()["n_det"]
        row = np.empty(n, np.int32)
        col = np.empty(n, np.int32)
        val = np.empty(n)
        self._check(self._L.mdet_get_ci_matrix(self._h, _ptr(row), _ptr(col), _ptr(val)), "mdet_get_ci_matrix")
        return row, col, val


def _ptr_array(vals):
    arr = (C.c_void_p * len(vals))()
    for i, v in enumerate(vals):
        arr[i] = v
    return arr


def _batch_args(ctxs, Rs, outs):
    n = len(ctxs)
    nw = (C.c_int64 * n)(*[int(R.shape[0]) for R in Rs])
    keys = ("log_abs_psi", "sign", "grad", "lap", "e_local", "status")
    cols = [_ptr_array([o[k].data_ptr() for o in outs]) for k in keys]
    return n, _ptr_array([c._h.value for c in ctxs]), nw, _ptr_array([R.data_ptr() for R in Rs]), cols


def batch_evaluate(ctxs, Rs, outs=None, n_streams=4, stream=None):
    """Evaluate several contexts (same device) on concurrent streams."""
    import torch
    if outs is None:
        outs = [c.alloc_outputs(R.shape[0]) for c, R in zip(ctxs, Rs)]
    if stream is None:
        stream = torch.cuda.current_stream(Rs[0].device)
    n, hs, nw, rp, cols = _batch_args(ctxs, Rs, outs)
    L = load_library()
    st = L.mdet_batch_evaluate(n, hs, nw, rp, *cols, int(n_streams), stream.cuda_stream)
    if st:
        raise MdetError(st, "mdet_batch_evaluate failed: %s" % L.mdet_status_string(st).decode())
    return outs


class Batch:
    """All evaluations of a list of contexts recorded once as a CUDA graph and
    replayed with one launch. The R tensors and outputs are baked in: refill R
    in place between launches."""

    def __init__(self, ctxs, Rs, outs=None, n_streams=4):
        if outs is None:
            outs = [c.alloc_outputs(R.shape[0]) for c, R in zip(ctxs, Rs)]
        self.ctxs, self.Rs, self.outs = list(ctxs), list(Rs), outs
        self._L = load_library()
        n, hs, nw, rp, cols = _batch_args(ctxs, Rs, outs)
        h = C.c_void_p()
        st = self._L.mdet_batch_create(C.byref(h), n, hs, nw, rp, *cols, int(n_streams))
        if st:
            raise MdetError(st, "mdet_batch_create failed: %s" % self._L.mdet_status_string(st).decode())
        self._h = h

    def launch(self, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.Rs[0].device)
        st = self._L.mdet_batch_launch(self._h, stream.cuda_stream)
        if st:
            raise MdetError(st, "mdet_batch_launch failed")
        return self.outs

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.mdet_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# VMC moves and the learned proposal

def _sp(stream, dev):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _chk(st, what):
    if st:
        raise MdetError(st, "%s failed: %s" % (what, load_library().mdet_status_string(st).decode()))


def gemm_bf16(A, B, D=None, accumulate=False, k_split=1024, stream=None):
    """D = bf16(A) bf16(B)^T on the tcgen05 tensor cores (FP32 accumulation): A [M][K] and
    B [N][K] FP32 CUDA tensors with unit inner stride; D [M][N] FP32, allocated when None.
    accumulate adds into D (atomics, K split over CTAs of k_split)."""
    import torch
    L = load_library()
    if A.dim() != 2 or B.dim() != 2 or A.shape[1] != B.shape[1]:
        raise ValueError("A [M][K] and B [N][K] expected")
    for t, name in ((A, "A"), (B, "B")):
        if t.dtype != torch.float32 or not t.is_cuda or t.stride(1) != 1:
            raise ValueError("%s: FP32 CUDA tensor with unit inner stride expected" % name)
    M, K = A.shape
    N = B.shape[0]
    if D is None:
        D = torch.zeros(M, N, dtype=torch.float32, device=A.device)
    elif D.shape != (M, N) or D.dtype != torch.float32 or D.stride(1) != 1 or D.device != A.device:
        raise ValueError("D: FP32 [M][N] tensor with unit inner stride on A's device expected")
    _chk(L.mdet_gemm_bf16(M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), D.data_ptr(), D.stride(0),
                          int(bool(accumulate)), int(k_split), _sp(stream, A.device)), "mdet_gemm_bf16")
    return D


def philox4x32_10(ctr, key):
    """Philox4x32-10 block for a 4-word counter and 2-word key (host)."""
    L = load_library()
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    L.mdet_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def _walkers(R):
    import torch
    if not (isinstance(R, torch.Tensor) and R.dim() == 3 and R.shape[2] == 3):
        raise ValueError("R must be a [n_walk, n_elec, 3] tensor")
    return R.shape[0], R.shape[1], R.device


def vmc_propose_drift(R, grad, tau, seed, step, R_new, log_q, stream=None):
    import torch
    W, N, dev = _walkers(R)
    for t, n in ((R, "R"), (grad, "grad"), (R_new, "R_new")):
        _need(t, n, (W, N, 3), torch.float64, dev)
    _need(log_q, "log_q", (W,), torch.float64, dev)
    _chk(load_library().mdet_vmc_propose_drift(R.shape[0], R.shape[1], R.data_ptr(), grad.data_ptr(), float(tau),
                                               int(seed), int(step), R_new.data_ptr(), log_q.data_ptr(),
                                               _sp(stream, R.device)), "mdet_vmc_propose_drift")


def vmc_reverse_drift(R, R_new, grad_new, tau, log_q, stream=None):
    import torch
    W, N, dev = _walkers(R)
    for t, n in ((R, "R"), (R_new, "R_new"), (grad_new, "grad_new")):
        _need(t, n, (W, N, 3), torch.float64, dev)
    _need(log_q, "log_q", (W,), torch.float64, dev)
    _chk(load_library().mdet_vmc_reverse_drift(R.shape[0], R.shape[1], R.data_ptr(), R_new.data_ptr(),
                                               grad_new.data_ptr(), float(tau), log_q.data_ptr(),
                                               _sp(stream, R.device)), "mdet_vmc_reverse_drift")


def vmc_accept(seed, step, log_q_fwd, log_q_rev, cur, new, accept=None, n_accept=None, stream=None):
    """cur / new: dicts with R, log_abs_psi, sign, grad, lap, e_local (device tensors)."""
    import torch
    R = cur["R"]
    W, N, dev = _walkers(R)
    for d, tag in ((cur, "cur"), (new, "new")):
        _need(d["R"], tag + "['R']", (W, N, 3), torch.float64, dev)
        _need(d["grad"], tag + "['grad']", (W, N, 3), torch.float64, dev)
        _need(d["lap"], tag + "['lap']", (W, N), torch.float64, dev)
        _need(d["sign"], tag + "['sign']", (W,), torch.int8, dev)
        for k in ("log_abs_psi", "e_local"):
            _need(d[k], "%s['%s']" % (tag, k), (W,), torch.float64, dev)
    for t, n in ((log_q_fwd, "log_q_fwd"), (log_q_rev, "log_q_rev")):
        _need(t, n, (W,), torch.float64, dev)
    if accept is not None:
        _need(accept, "accept", (W,), torch.int32, dev)
    if n_accept is not None:
        _need(n_accept, "n_accept", (1,), torch.int32, dev)
    _chk(load_library().mdet_vmc_accept(
        R.shape[0], R.shape[1], int(seed), int(step), log_q_fwd.data_ptr(), log_q_rev.data_ptr(), R.data_ptr(),
        cur["log_abs_psi"].data_ptr(), cur["sign"].data_ptr(), cur["grad"].data_ptr(), cur["lap"].data_ptr(),
        cur["e_local"].data_ptr(), new["R"].data_ptr(), new["log_abs_psi"].data_ptr(), new["sign"].data_ptr(),
        new["grad"].data_ptr(), new["lap"].data_ptr(), new["e_local"].data_ptr(),
        accept.data_ptr() if accept is not None else None, n_accept.data_ptr() if n_accept is not None else None,
        _sp(stream, R.device)), "mdet_vmc_accept")


def vmc_limit_drift(F, tau, a, F_bar, stream=None):
    """Per-electron drift limiting (Umrigar, Nightingale and Runge); a = 0 copies F."""
    import torch
    W, N, dev = _walkers(F)
    _need(F, "F", (W, N, 3), torch.float64, dev)
    _need(F_bar, "F_bar", (W, N, 3), torch.float64, dev)
    _chk(load_library().mdet_vmc_limit_drift(F.shape[0], F.shape[1], F.data_ptr(), float(tau), float(a),
                                             F_bar.data_ptr(), _sp(stream, F.device)), "mdet_vmc_limit_drift")


def vmc_select_rows(take, src, dst, stream=None):
    """dst[w] = src[w] where take[w] != 0 (float32 rows)."""
    import torch
    if not (isinstance(src, torch.Tensor) and src.dim() == 2):
        raise ValueError("src must be a [n_walk, width] tensor")
    _need(src, "src", tuple(src.shape), torch.float32, src.device)
    _need(dst, "dst", tuple(src.shape), torch.float32, src.device)
    _need(take, "take", (src.shape[0],), torch.int32, src.device)
    _chk(load_library().mdet_vmc_select_rows(src.shape[0], src.shape[1], take.data_ptr(), src.data_ptr(),
                                             dst.data_ptr(), _sp(stream, src.device)), "mdet_vmc_select_rows")


def vmc_r2(R, r2, stream=None):
    import torch
    W, N, dev = _walkers(R)
    _need(R, "R", (W, N, 3), torch.float64, dev)
    _need(r2, "r2", (W,), torch.float64, dev)
    _chk(load_library().mdet_vmc_r2(R.shape[0], R.shape[1], R.data_ptr(), r2.data_ptr(), _sp(stream, R.device)),
         "mdet_vmc_r2")


class MLP:
    """The learned proposal's perceptron (3N -> H -> H -> 4N, tanh, BF16 weights, FP32 accumulation)."""

    def __init__(self, device, n_elec, hidden=256, seed=1, mu_max=1.0, s0=-1.5, s_span=2.0, coord_scale=2.0,
                 langevin=True, zero_head=True):
        """langevin: moves take the Langevin form (mean R + mu + sigma^2 F, F the
        drift at R); zero_head: the output layer starts at zero, so that the
        untrained proposal is the drift-diffusion move with tau = exp(2 s0)
        (langevin) or an isotropic Gaussian of scale exp(s0)."""
        self._L = load_library()
        h = C.c_void_p()
        _chk(self._L.mdet_mlp_create(C.byref(h), int(device), int(n_elec), int(hidden), int(seed), float(mu_max),
                                     float(s0), float(s_span), float(coord_scale)), "mdet_mlp_create")
        self._h = h
        self.device, self.n_elec, self.hidden = int(device), int(n_elec), int(hidden)
        self.mu_max, self.s0, self.s_span, self.coord_scale = mu_max, s0, s_span, coord_scale
        self.n_params = int(self._L.mdet_mlp_n_params(h))
        self.langevin = bool(langevin)
        if zero_head:
            p = self.params()
            n_in, H, n_out = 3 * self.n_elec, self.hidden, 4 * self.n_elec
            p[n_in * H + H + H * H + H:] = 0.0
            self.set_params(p)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.mdet_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        p = np.empty(self.n_params, np.float32)
        _chk(self._L.mdet_mlp_get_params(self._h, _ptr(p)), "mdet_mlp_get_params")
        return p

    def set_params(self, p):
        p = _c(p, np.float32)
        _chk(self._L.mdet_mlp_set_params(self._h, _ptr(p)), "mdet_mlp_set_params")

    def grads(self):
        g = np.empty(self.n_params, np.float32)
        _chk(self._L.mdet_mlp_get_grads(self._h, _ptr(g)), "mdet_mlp_get_grads")
        return g

    def _pos(self, R, name="R"):
        """(n_walk, device) of a position tensor [n_walk, n_elec, 3] float64 on this network's device."""
        import torch
        dev = torch.device("cuda", self.device)
        n = R.shape[0] if isinstance(R, torch.Tensor) and R.dim() == 3 else -1
        _need(R, name, (n, self.n_elec, 3), torch.float64, dev)
        return n, dev

    def _outs(self, n, dev, **tensors):
        import torch
        for name, t in tensors.items():
            _need(t, name, (n, 4 * self.n_elec), torch.float32, dev)

    def forward(self, R, out=None, stream=None):
        import torch
        n, dev = self._pos(R)
        if out is None:
            out = torch.empty(n, 4 * self.n_elec, dtype=torch.float32, device=dev)
        self._outs(n, dev, out=out)
        _chk(self._L.mdet_mlp_forward(self._h, n, R.data_ptr(), out.data_ptr(), _sp(stream, dev)),
             "mdet_mlp_forward")
        self._last_n = n
        return out

    def backward(self, dout, stream=None):
        """Backward pass of the last forward (dout has its walker count)."""
        import torch
        dev = torch.device("cuda", self.device)
        n = getattr(self, "_last_n", None)
        if n is None:
            raise ValueError("backward needs a forward pass first")
        self._outs(n, dev, dout=dout)
        _chk(self._L.mdet_mlp_backward(self._h, n, dout.data_ptr(), _sp(stream, dev)), "mdet_mlp_backward")

    def zero_grad(self, stream=None):
        import torch
        _chk(self._L.mdet_mlp_zero_grad(self._h, _sp(stream, torch.device("cuda", self.device))), "mdet_mlp_zero_grad")

    def adam(self, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        import torch
        _chk(self._L.mdet_mlp_adam(self._h, float(lr), float(beta1), float(beta2), float(eps), int(t),
                                   _sp(stream, torch.device("cuda", self.device))), "mdet_mlp_adam")

    def nll_grad(self, R0, R1, out, dout, loss, stream=None):
        import torch
        n, dev = self._pos(R0, "R0")
        _need(R1, "R1", (n, self.n_elec, 3), torch.float64, dev)
        self._outs(n, dev, out=out, dout=dout)
        _need(loss, "loss", (1,), torch.float64, dev)
        _chk(self._L.mdet_mlp_nll_grad(self._h, R0.shape[0], R0.data_ptr(), R1.data_ptr(), out.data_ptr(),
                                       dout.data_ptr(), loss.data_ptr(), _sp(stream, R0.device)), "mdet_mlp_nll_grad")

    def esjd_grad(self, R, R_new, out, out_new, log_abs_psi, log_abs_psi_new, sign_new, drift, drift_new,
                  grad_new, dout, dout_new, objective, jump_len2=0.0, speed_beta=0.0, stream=None):
        """drift, drift_new: the drift arrays of the forward move and the reverse
        density (e.g. limited); grad_new: grad Psi / Psi at R_new; objective: two
        device doubles (J, mean acceptance); speed_beta > 0 selects the speed measure."""
        import torch
        lg = self.langevin
        n, dev = self._pos(R)
        for t, name in ((R_new, "R_new"), (grad_new, "grad_new")) + (((drift, "drift"), (drift_new, "drift_new"))
                                                                   if lg else ()):
            _need(t, name, (n, self.n_elec, 3), torch.float64, dev)
        self._outs(n, dev, out=out, out_new=out_new, dout=dout, dout_new=dout_new)
        _need(log_abs_psi, "log_abs_psi", (n,), torch.float64, dev)
        _need(log_abs_psi_new, "log_abs_psi_new", (n,), torch.float64, dev)
        _need(sign_new, "sign_new", (n,), torch.int8, dev)
        _need(objective, "objective", (2,), torch.float64, dev)
        _chk(self._L.mdet_mlp_esjd_grad(self._h, R.shape[0], R.data_ptr(), R_new.data_ptr(), out.data_ptr(),
                                        out_new.data_ptr(), log_abs_psi.data_ptr(), log_abs_psi_new.data_ptr(),
                                        sign_new.data_ptr(), drift.data_ptr() if lg else None,
                                        drift_new.data_ptr() if lg else None, grad_new.data_ptr(), int(lg),
                                        float(jump_len2), float(speed_beta), dout.data_ptr(),
                                        dout_new.data_ptr(), objective.data_ptr(), _sp(stream, R.device)),
             "mdet_mlp_esjd_grad")

    def propose(self, R, out, seed, step, R_new, log_q, drift=None, stream=None):
        """drift: grad Psi / Psi at R, required for the Langevin form."""
        import torch
        if self.langevin and drift is None:
            raise ValueError("the Langevin form needs the drift at R")
        n, dev = self._pos(R)
        _need(R_new, "R_new", (n, self.n_elec, 3), torch.float64, dev)
        if self.langevin:
            _need(drift, "drift", (n, self.n_elec, 3), torch.float64, dev)
        self._outs(n, dev, out=out)
        _need(log_q, "log_q", (n,), torch.float64, dev)
        _chk(self._L.mdet_vmc_propose_mlp(self._h, R.shape[0], R.data_ptr(), out.data_ptr(),
                                          drift.data_ptr() if self.langevin else None, int(seed), int(step),
                                          R_new.data_ptr(), log_q.data_ptr(), _sp(stream, R.device)),
             "mdet_vmc_propose_mlp")

    def reverse(self, R, R_new, out_new, log_q, drift_new=None, stream=None):
        """drift_new: grad Psi / Psi at R_new, required for the Langevin form."""
        import torch
        if self.langevin and drift_new is None:
            raise ValueError("the Langevin form needs the drift at R_new")
        n, dev = self._pos(R)
        _need(R_new, "R_new", (n, self.n_elec, 3), torch.float64, dev)
        if self.langevin:
            _need(drift_new, "drift_new", (n, self.n_elec, 3), torch.float64, dev)
        self._outs(n, dev, out_new=out_new)
        _need(log_q, "log_q", (n,), torch.float64, dev)
        _chk(self._L.mdet_vmc_reverse_mlp(self._h, R.shape[0], R.data_ptr(), R_new.data_ptr(), out_new.data_ptr(),
                                          drift_new.data_ptr() if self.langevin else None, log_q.data_ptr(),
                                          _sp(stream, R.device)), "mdet_vmc_reverse_mlp")
