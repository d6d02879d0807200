"""Thin ctypes binding of liblrnr.so (C ABI in ``include/lrnr.h``).

Each function has the name of the C entry point it wraps and only marshals
arguments: torch tensors are passed as device pointers, host arrays as FP64
buffers.  All computation happens in the library's CUDA kernels; if the library
is missing the import fails loudly (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblrnr.so")

OK, EINVAL, ENOMEM, ECUDA, ESINGULAR, EEARLYSTOP, ETIMEOUT, ENOTREADY, ENONFINITE, ENOTSUP, ETOOBIG = range(11)
FP32, TF32, BF16, BF16X3 = 0, 1, 2, 3
FULL, FAST = 0, 1
LOSS_MSE, LOSS_L1 = 0, 1

_PREC = {"fp32": FP32, "tf32": TF32, "bf16": BF16, "bf16x3": BF16X3}
_FORM = {"full": FULL, "fast": FAST}
_LOSS = {"mse": LOSS_MSE, "l1": LOSS_L1}


class LrnrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {lrnr_status_string(status)} (status {status})")


class lrnr_batch(ctypes.Structure):
    _fields_ = [
        ("n_inst", ctypes.c_int32),
        ("n_int", ctypes.c_int64), ("n_ic", ctypes.c_int64), ("n_bc", ctypes.c_int64),
        ("beta", ctypes.c_void_p), ("nu", ctypes.c_void_p), ("rho", ctypes.c_void_p),
        ("s", ctypes.c_void_p),
        ("int_off", ctypes.c_void_p), ("ic_off", ctypes.c_void_p), ("bc_off", ctypes.c_void_p),
        ("x_int", ctypes.c_void_p), ("t_int", ctypes.c_void_p),
        ("x_ic", ctypes.c_void_p), ("t_bc", ctypes.c_void_p),
        ("norm", ctypes.c_void_p),
    ]


_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "lrnr_build": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "lrnr_snapshots": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, _P, _P, ctypes.c_int, _P, _P, _P]),
    "fastlrnr_select_rows": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int64, ctypes.c_int,
                                            ctypes.c_double, _P, _P, _P, _P, _P, _P]),
    "lrnr_residual": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "lrnr_residual_grad": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P,
                                          _P, _P, _P, _P]),
    "spinprop_step": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P,
                                     _P, _P, _P, _P, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_float, ctypes.c_float, _P, _P, _P]),
    "lrnr_residual_grad_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, _P, _P, _P]),
    "lrnr_adam_update": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, _P,
                                        ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_float, ctypes.c_float, _P, _P, _P, _P]),
    "lrnr_copy_pinned": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "lrnr_reserve": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32]),
    "lrnr_model_info": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "lrnr_set_tuning": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "lrnr_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "lrnr_timing_read": (ctypes.c_int, [_P, _P, _P]),
    "lrnr_last_device_status": (ctypes.c_int, [_P]),
    "lrnr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lrnr_destroy": (None, [_P]),
    "lrnr_measure_peaks": (ctypes.c_int, [_P, _P]),
    "lrnr_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_int64]),
    "lrnr_pod": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                ctypes.c_double, _P, _P, _P, _P, _P]),
    "lrnr_deim_rows": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
}

EXPORTS = tuple(_SIGS)


def lib():
    """Load liblrnr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"liblrnr.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != OK:
        raise LrnrError(rc, where)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensors passed to liblrnr must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    return t


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def lrnr_status_string(status: int) -> str:
    return lib().lrnr_status_string(int(status)).decode()


class Model:
    """Owns an ``lrnr_model *``; destroyed with :func:`lrnr_destroy` or on GC."""

    def __init__(self, handle, L, M, r):
        self.handle = handle
        self.L, self.M, self.r = L, M, list(r)
        self.sum_r = int(sum(r))
        self.sum_m = L * M + 1

    def __del__(self):
        try:
            lrnr_destroy(self)
        except Exception:
            pass


def lrnr_build(L: int, M: int, r, U, V, b) -> Model:
    """Create a model from FP64 host bases (lists of L+1 row-major arrays)."""
    keep = []

    def ptrs(mats):
        arr = (ctypes.c_void_p * len(mats))()
        for i, a in enumerate(mats):
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            arr[i] = a.ctypes.data
        return arr

    rr = (ctypes.c_int * len(r))(*[int(v) for v in r])
    out = ctypes.c_void_p()
    rc = lib().lrnr_build(int(L), int(M), ctypes.cast(rr, _P), ctypes.cast(ptrs(U), _P),
                          ctypes.cast(ptrs(V), _P), ctypes.cast(ptrs(b), _P), ctypes.byref(out))
    _check(rc, "lrnr_build")
    return Model(out, L, M, r)


def lrnr_destroy(model: Model):
    if model.handle:
        lib().lrnr_destroy(model.handle)
        model.handle = None


def lrnr_reserve(model: Model, max_points: int, max_inst: int):
    _check(lib().lrnr_reserve(model.handle, int(max_points), int(max_inst)), "lrnr_reserve")


def lrnr_model_info(model: Model) -> dict:
    v = [ctypes.c_int() for _ in range(5)]
    _check(lib().lrnr_model_info(model.handle, *[ctypes.byref(x) for x in v]), "lrnr_model_info")
    return dict(zip(("L", "M", "sum_r", "sum_m", "fast_ready"), [x.value for x in v]))


def lrnr_set_tuning(model: Model, form: str, prec: str, nt: int = 0, ctas_per_sm: int = 0):
    """Override the launch shape for (form, prec); 0 = automatic."""
    _check(lib().lrnr_set_tuning(model.handle, _FORM[form], _PREC[prec], int(nt), int(ctas_per_sm)),
           "lrnr_set_tuning")


def lrnr_set_wait_limit(model: Model, polls: int = -1):
    """Iteration cap of the tensor-core kernel's waits (polls per wait; -1 = default)."""
    _check(lib().lrnr_set_wait_limit(model.handle, int(polls)), "lrnr_set_wait_limit")


def lrnr_timing(model: Model, enable: bool = True):
    _check(lib().lrnr_timing(model.handle, int(bool(enable))), "lrnr_timing")


def lrnr_timing_read(model: Model):
    """(summed tile-kernel milliseconds, launches) since the last read."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(lib().lrnr_timing_read(model.handle, ctypes.byref(ms), ctypes.byref(n)), "lrnr_timing_read")
    return ms.value, n.value


class lrnr_peaks(ctypes.Structure):
    _fields_ = [("fp32_fma_tflops", ctypes.c_double), ("fp32_fma2_tflops", ctypes.c_double),
                ("tanh_approx_gops", ctypes.c_double), ("tanhf_gops", ctypes.c_double),
                ("fp64_fma_tflops", ctypes.c_double), ("sm_mhz", ctypes.c_double),
                ("sms", ctypes.c_int)]


def lrnr_measure_peaks(stream=None) -> dict:
    """Compute-throughput microbenchmarks of the current device (see include/lrnr.h)."""
    out = lrnr_peaks()
    _check(lib().lrnr_measure_peaks(ctypes.byref(out), _stream(stream)), "lrnr_measure_peaks")
    return {name: getattr(out, name) for name, _ in lrnr_peaks._fields_}


def lrnr_last_device_status(model: Model) -> int:
    return int(lib().lrnr_last_device_status(model.handle))


class DeviceBatch:
    """Device copies of a batch (float32 points and parameters, int64 offsets) and
    the ``lrnr_batch`` struct that points at them.  ``norm`` (optional, int64
    (n_inst, 3)): the MSE denominators of each instance (interior, initial,
    periodic), for a batch that holds one shard of the instances' points."""

    def __init__(self, n_inst, beta, nu, rho, s, int_off, ic_off, bc_off, x_int, t_int, x_ic, t_bc,
                 norm=None):
        self.tensors = dict(beta=beta, nu=nu, rho=rho, s=s, int_off=int_off, ic_off=ic_off,
                            bc_off=bc_off, x_int=x_int, t_int=t_int, x_ic=x_ic, t_bc=t_bc)
        for k, v in self.tensors.items():
            setattr(self, k, v)
        self.norm = norm
        self.n_inst = n_inst
        self.struct = lrnr_batch()
        self.refresh()

    def refresh(self):
        st = self.struct
        st.n_inst = self.n_inst
        st.n_int = int(self.x_int.numel())
        st.n_ic = int(self.x_ic.numel())
        st.n_bc = int(self.t_bc.numel())
        for k in ("beta", "nu", "rho", "s", "int_off", "ic_off", "bc_off", "x_int", "t_int", "x_ic", "t_bc"):
            t = getattr(self, k)
            setattr(st, k, t.data_ptr() if t is not None and t.numel() else None)
        if self.norm is not None:
            if self.norm.dtype != torch.int64 or tuple(self.norm.shape) != (self.n_inst, 3) \
                    or not self.norm.is_contiguous():
                raise ValueError("norm must be a contiguous int64 tensor of shape (n_inst, 3)")
            st.norm = self.norm.data_ptr()
        else:
            st.norm = None

    def with_s(self, s):
        """A batch sharing these points but reading coefficients from ``s``."""
        t = dict(self.tensors)
        t["s"] = s
        return DeviceBatch(self.n_inst, **t, norm=self.norm)

    @property
    def n_points(self) -> int:
        return int(self.x_int.numel() + self.x_ic.numel() + 2 * self.t_bc.numel())

    @classmethod
    def from_host(cls, bt, device="cuda", s=None, pin=False, norm=None):
        f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32))
        i64 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.int64))
        host = dict(beta=f32(bt.beta), nu=f32(bt.nu), rho=f32(bt.rho),
                    s=f32(bt.s if s is None else s), int_off=i64(bt.int_off), ic_off=i64(bt.ic_off),
                    bc_off=i64(bt.bc_off), x_int=f32(bt.x_int), t_int=f32(bt.t_int),
                    x_ic=f32(bt.x_ic), t_bc=f32(bt.t_bc))
        if pin:
            host = {k: v.pin_memory() for k, v in host.items()}
        dev = {k: v.to(device, non_blocking=pin) for k, v in host.items()}
        nd = None if norm is None else torch.as_tensor(
            np.ascontiguousarray(norm, dtype=np.int64)).to(device)
        return cls(bt.n_inst, **dev, norm=nd)


def lrnr_snapshots(model: Model, layer: int, x, t, s, stream=None):
    """FP64 exact-LRNR states of hidden layer ``layer``: (M, n_s * n_pts) column-major,
    returned as a tensor of shape (n_s * n_pts, M)."""
    x = x.to(torch.float64).contiguous()
    t = t.to(torch.float64).contiguous()
    s = s.to(torch.float64).contiguous().reshape(-1, model.sum_r)
    out = torch.empty((s.shape[0] * x.numel(), model.M), dtype=torch.float64, device=x.device)
    rc = lib().lrnr_snapshots(model.handle, int(layer), int(x.numel()), _ptr(x), _ptr(t),
                              int(s.shape[0]), _ptr(s), _ptr(out), _stream(stream))
    _check(rc, "lrnr_snapshots")
    return out


def fastlrnr_select_rows(model: Model, layer: int, snapshots=None, rhat: int = 16, tol: float = 0.0,
                         rows_in=None, Xi_in=None, stream=None):
    """EIM selection for one hidden layer.  ``snapshots``: device FP64 tensor of shape
    (K, M) (row k = snapshot k, i.e. the column-major M x K matrix).  Returns
    (rows int32 tensor, Xi tensor of shape (rhat_used, M), rhat_used)."""
    dev = snapshots.device if snapshots is not None else rows_in.device
    rows = torch.full((rhat,), -1, dtype=torch.int32, device=dev)
    Xi = torch.zeros((rhat, model.M), dtype=torch.float64, device=dev)
    used = ctypes.c_int(0)
    K = 0 if snapshots is None else int(snapshots.shape[0])
    if snapshots is not None:
        snapshots = snapshots.contiguous()
    if rows_in is not None:
        rows_in = rows_in.to(torch.int32).contiguous()
        Xi_in = Xi_in.to(torch.float64).contiguous()
    rc = lib().fastlrnr_select_rows(model.handle, int(layer), _ptr(snapshots), K, int(rhat),
                                    float(tol), _ptr(rows_in), _ptr(Xi_in), _ptr(rows), _ptr(Xi),
                                    ctypes.byref(used), _stream(stream))
    _check(rc, "fastlrnr_select_rows")
    n = used.value
    return rows[:n], Xi[:n], n


def lrnr_pod(snapshots, n_modes: int, n_iter: int = 30, tol: float = 1e-10, stream=None):
    """POD modes of a snapshot matrix.  ``snapshots``: device FP64 tensor of shape
    (K, M) (the column-major M x K matrix).  Returns (Xi of shape (n_used, M), i.e.
    the column-major M x n_used basis, sigma (n_used,), resid (n_used,), n_used)."""
    S = snapshots.to(torch.float64).contiguous()
    K, M = int(S.shape[0]), int(S.shape[1])
    n = min(int(n_modes), M, K)
    Xi = torch.zeros((n, M), dtype=torch.float64, device=S.device)
    sig = torch.zeros(n, dtype=torch.float64, device=S.device)
    res = torch.zeros(n, dtype=torch.float64, device=S.device)
    used = ctypes.c_int(0)
    rc = lib().lrnr_pod(_ptr(S), M, K, int(n_modes), int(n_iter), float(tol), _ptr(Xi), _ptr(sig),
                        _ptr(res), ctypes.byref(used), _stream(stream))
    _check(rc, "lrnr_pod")
    u = used.value
    return Xi[:u], sig[:u], res[:u], u


def lrnr_deim_rows(Xi, stream=None):
    """DEIM rows of the basis ``Xi`` (device FP64, shape (n, M): column-major M x n)."""
    Xi = Xi.to(torch.float64).contiguous()
    n, M = int(Xi.shape[0]), int(Xi.shape[1])
    rows = torch.full((n,), -1, dtype=torch.int32, device=Xi.device)
    rc = lib().lrnr_deim_rows(_ptr(Xi), M, n, _ptr(rows), _stream(stream))
    _check(rc, "lrnr_deim_rows")
    return rows


def fastlrnr_select_rows_deim(model: Model, layer: int, snapshots, rhat: int = 16,
                              n_iter: int = 30, tol: float = 1e-10, stream=None):
    """DEIM selection for one hidden layer: POD basis of the snapshots (``lrnr_pod``),
    its DEIM rows (``lrnr_deim_rows``), then the reduced layer of Eq. 2.7 installed
    through ``fastlrnr_select_rows`` with those rows and that basis.  Returns
    (rows, Xi of shape (rhat_used, M), rhat_used, sigma)."""
    Xi, sig, _, used = lrnr_pod(snapshots, rhat, n_iter=n_iter, tol=tol, stream=stream)
    if used < 1:
        raise LrnrError(4, "lrnr_pod: no mode above the cut")
    rows = lrnr_deim_rows(Xi, stream=stream)
    rows, Xi, used = fastlrnr_select_rows(model, layer, None, used, 0.0, rows_in=rows, Xi_in=Xi,
                                          stream=stream)
    return rows, Xi, used, sig


def lrnr_residual(model: Model, form: str, prec: str, batch: DeviceBatch, stream=None, out=None):
    """Forward only: dict with u, u_t, u_x, u_xx, res (interior), res_ic, res_bc."""
    dev = batch.x_int.device
    if out is None:
        ni, nc, nb = batch.x_int.numel(), batch.x_ic.numel(), batch.t_bc.numel()
        out = {k: torch.empty(ni, dtype=torch.float32, device=dev) for k in ("u", "u_t", "u_x", "u_xx", "res")}
        out["res_ic"] = torch.empty(nc, dtype=torch.float32, device=dev)
        out["res_bc"] = torch.empty(nb, dtype=torch.float32, device=dev)
    rc = lib().lrnr_residual(model.handle, _FORM[form], _PREC[prec], ctypes.byref(batch.struct),
                             *[_ptr(out.get(k)) for k in ("u", "u_t", "u_x", "u_xx", "res", "res_ic", "res_bc")],
                             _stream(stream))
    _check(rc, "lrnr_residual")
    return out


def lrnr_residual_grad(model: Model, form: str, prec: str, batch: DeviceBatch, loss: str = "mse",
                       w=None, want_db: bool = True, stream=None, out=None):
    """Loss (n_inst,), dL/ds (n_inst, sum_r), dL/db (n_inst, sum_m) or None."""
    dev = batch.x_int.device
    if out is None:
        out = (torch.empty(batch.n_inst, dtype=torch.float32, device=dev),
               torch.empty((batch.n_inst, model.sum_r), dtype=torch.float32, device=dev),
               torch.empty((batch.n_inst, model.sum_m), dtype=torch.float32, device=dev) if want_db else None)
    wa = None if w is None else (ctypes.c_float * 3)(*[float(v) for v in w])
    rc = lib().lrnr_residual_grad(model.handle, _FORM[form], _PREC[prec], ctypes.byref(batch.struct),
                                  _LOSS[loss], ctypes.cast(wa, _P) if wa is not None else None,
                                  _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _stream(stream))
    _check(rc, "lrnr_residual_grad")
    return out


def lrnr_residual_grad_noalloc(model: Model, batch: DeviceBatch, loss: str = "mse", w=None,
                               want_db: bool = True, stream=None, out=None):
    """FastLRNR FP32 loss and gradient computed without any device allocation: the
    library's fixed 32 MiB scratch replaces the model workspace (for callers whose
    device memory belongs to another allocator or a fixed budget).  Output buffers
    are still the caller's; pass ``out`` to reuse them."""
    dev = batch.x_int.device
    if out is None:
        out = (torch.empty(batch.n_inst, dtype=torch.float32, device=dev),
               torch.empty((batch.n_inst, model.sum_r), dtype=torch.float32, device=dev),
               torch.empty((batch.n_inst, model.sum_m), dtype=torch.float32, device=dev) if want_db else None)
    wa = None if w is None else (ctypes.c_float * 3)(*[float(v) for v in w])
    rc = lib().lrnr_residual_grad_noalloc(model.handle, ctypes.byref(batch.struct), _LOSS[loss],
                                          ctypes.cast(wa, _P) if wa is not None else None,
                                          _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _stream(stream))
    _check(rc, "lrnr_residual_grad_noalloc")
    return out


def spinprop_step(model: Model, form: str, prec: str, batch: DeviceBatch, s, m, v, step,
                  n_steps: int = 1, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
                  eps: float = 1e-8, lambda_loc: float = 0.0, s_anchor=None, loss: str = "mse",
                  w=None, loss_out=None, stream=None):
    """``n_steps`` fused residual + gradient + Adam steps on ``s`` (in place)."""
    wa = None if w is None else (ctypes.c_float * 3)(*[float(x) for x in w])
    rc = lib().spinprop_step(model.handle, _FORM[form], _PREC[prec], ctypes.byref(batch.struct),
                             _LOSS[loss], ctypes.cast(wa, _P) if wa is not None else None,
                             _ptr(s), _ptr(m), _ptr(v), _ptr(step), int(n_steps), float(lr),
                             float(beta1), float(beta2), float(eps), float(lambda_loc),
                             _ptr(s_anchor), _ptr(loss_out), _stream(stream))
    _check(rc, "spinprop_step")
    return s


def lrnr_adam_update(grad, s, m, v, step, lr: float = 1e-3, beta1: float = 0.9,
                     beta2: float = 0.999, eps: float = 1e-8, lambda_loc: float = 0.0,
                     s_anchor=None, loss_in=None, loss_out=None, stream=None):
    """One Adam step on ``s`` (in place) from the gradient ``grad`` (n_inst, sum_r),
    advancing the device step counter ``step``; ``loss_out`` = ``loss_in`` plus the
    locality term."""
    n_inst, sum_r = (int(grad.shape[0]), int(grad.shape[1])) if grad.dim() == 2 else (1, int(grad.numel()))
    rc = lib().lrnr_adam_update(n_inst, sum_r, _ptr(grad), _ptr(s), _ptr(m), _ptr(v), _ptr(step),
                                float(lr), float(beta1), float(beta2), float(eps), float(lambda_loc),
                                _ptr(s_anchor), _ptr(loss_in), _ptr(loss_out), _stream(stream))
    _check(rc, "lrnr_adam_update")
    return s


def lrnr_copy_pinned(dst, src, stream=None):
    """Copy tensor ``src`` into ``dst`` (same number of bytes, both contiguous) with the
    library's copy kernel; each side is a CUDA tensor of the current device or a pinned
    CPU tensor.  Stream-ordered: a CPU destination holds the result once the stream has
    been synchronised."""
    nb = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() != nb:
        raise ValueError("lrnr_copy_pinned: dst and src differ in size")
    if nb == 0:
        return dst
    for t in (dst, src):
        if t.device.type == "cpu" and not t.is_pinned():
            raise ValueError("lrnr_copy_pinned: CPU tensors must be pinned")
    _check(lib().lrnr_copy_pinned(_ptr(dst), _ptr(src), nb, _stream(stream)), "lrnr_copy_pinned")
    return dst
