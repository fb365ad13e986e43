"""ctypes binding of liblqcd.so (the C ABI in include/lqcd.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  The raw entry points keep their C names (``lqcd_create``,
``lqcd_deo_apply``, ``lqcd_mscg_solve`` ...); ``Context`` and ``Server`` wrap
them with numpy / torch arguments and raise ``LqcdError`` on a non-zero
status.  Loading fails loudly when the library is missing: there is no CPU
fallback.

Device spinors are torch tensors in the library's structure-of-arrays layout:
complex128 (or complex64 for FP32/FP16 calls) of shape ``[3, Vh]`` (one
field) or ``[n, 3, Vh]`` (several fields); ``to_device_spinor`` /
``from_device_spinor`` convert from / to the canonical host ``[Vh, 3]``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblqcd.so")

LQCD_OK = 0
LQCD_EINVAL = -1
LQCD_ENOMEM = -2
LQCD_ENOCONV = -3
LQCD_ENAN = -4
LQCD_EBUSY = -5
LQCD_ENOTREADY = -6
LQCD_ETIMEOUT = -7
LQCD_ECUDA = -8
LQCD_ESTATE = -9
STATUS_NAMES = {0: "LQCD_OK", -1: "LQCD_EINVAL", -2: "LQCD_ENOMEM", -3: "LQCD_ENOCONV", -4: "LQCD_ENAN",
                -5: "LQCD_EBUSY", -6: "LQCD_ENOTREADY", -7: "LQCD_ETIMEOUT", -8: "LQCD_ECUDA",
                -9: "LQCD_ESTATE"}

PREC_FP64, PREC_FP32, PREC_FP16, PREC_FP64_NATIVE = 0, 1, 2, 3
MAX_SHIFTS = 32

# Every symbol include/lqcd.h declares (checked by the CPU tests).
EXPORTED = [
    "lqcd_default_opts", "lqcd_last_error", "lqcd_version", "lqcd_create", "lqcd_destroy",
    "lqcd_set_opts", "lqcd_device_bytes", "lqcd_links_upload", "lqcd_links_download",
    "lqcd_deo_apply", "lqcd_deo_apply_host_noalloc", "lqcd_deo_apply_ex", "lqcd_deo_apply_mrhs", "lqcd_mscg_solve",
    "lqcd_mscg_solve_dev", "lqcd_rational_apply", "lqcd_rational_apply_dev", "lqcd_cg_solve_mrhs",
    "lqcd_mscg_solve_packed", "lqcd_profile_iteration",
    "lqcd_serve_create", "lqcd_serve_register_field", "lqcd_serve_submit", "lqcd_serve_poll",
    "lqcd_serve_drain", "lqcd_serve_stats_get", "lqcd_serve_destroy", "lqcd_serve_set_opts",
    "lqcd_mom_upload", "lqcd_mom_download", "lqcd_gauge_mom_update", "lqcd_gauge_link_update",
    "lqcd_gauge_md_steps", "lqcd_gauge_action", "lqcd_mom_energy", "lqcd_fermion_force_update",
    "lqcd_stout_smear", "lqcd_stout_restore", "lqcd_stout_force", "lqcd_deo_apply_mrhs_layout",
    "lqcd_selftest_stage_wait", "lqcd_inject_alloc_failure", "lqcd_bounds_errors",
    "lqcd_shard_create", "lqcd_shard_geometry", "lqcd_shard_links_upload", "lqcd_shard_deo_apply",
    "lqcd_shard_exchange", "lqcd_shard_cg_solve", "lqcd_deo_tuned_config",
    "lqcd_measure_fma_rates", "lqcd_deo_apply_h16",
]


class lqcd_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("recon", ctypes.c_int), ("delta_reliable", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("check_every", ctypes.c_int), ("fp64_until", ctypes.c_double),
                ("staged", ctypes.c_int), ("pdl", ctypes.c_int)]


class lqcd_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("n_shift", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("refine_iters", ctypes.c_int), ("shift_iters", ctypes.c_int * MAX_SHIFTS),
                ("true_resid", ctypes.c_double * MAX_SHIFTS), ("secs", ctypes.c_double),
                ("bytes_moved", ctypes.c_double), ("status", ctypes.c_int), ("kernel_launches", ctypes.c_int)]

    def as_dict(self) -> dict:
        n = self.n_shift
        return {"iters": self.iters, "n_shift": n, "reliable_updates": self.reliable_updates,
                "refine_iters": self.refine_iters, "shift_iters": list(self.shift_iters)[:n],
                "true_resid": list(self.true_resid)[:n], "secs": self.secs,
                "bytes_moved": self.bytes_moved, "status": self.status,
                "kernel_launches": self.kernel_launches}


class lqcd_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("active_slots", ctypes.c_int), ("queued", ctypes.c_int), ("hbm_in_use", ctypes.c_size_t),
                ("hbm_budget", ctypes.c_size_t), ("p50_latency", ctypes.c_double),
                ("p99_latency", ctypes.c_double), ("mean_latency", ctypes.c_double),
                ("solves_per_sec", ctypes.c_double), ("ticks", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class LqcdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load liblqcd.so (build it first with paper_1701_00426_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"liblqcd.so not found at {p}: run paper_1701_00426_gb300.build.build() "
                          f"(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(p)
    vp, ip, dp, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.c_size_t
    sig = {
        "lqcd_default_opts": (None, [ctypes.POINTER(lqcd_opts)]),
        "lqcd_last_error": (ctypes.c_char_p, []),
        "lqcd_version": (ctypes.c_int, []),
        "lqcd_create": (ctypes.c_int, [ip, ctypes.POINTER(lqcd_opts), ctypes.POINTER(vp)]),
        "lqcd_destroy": (None, [vp]),
        "lqcd_set_opts": (ctypes.c_int, [vp, ctypes.POINTER(lqcd_opts)]),
        "lqcd_device_bytes": (sz, [vp]),
        "lqcd_links_upload": (ctypes.c_int, [vp, vp, sz]),
        "lqcd_links_download": (ctypes.c_int, [vp, vp, sz]),
        "lqcd_deo_apply": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, ctypes.c_int, vp]),
        "lqcd_deo_apply_host_noalloc": (ctypes.c_int, [vp, ctypes.c_int, vp, vp]),
        "lqcd_deo_apply_ex": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp]),
        "lqcd_deo_apply_mrhs": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp]),
        "lqcd_mscg_solve": (ctypes.c_int, [vp, ctypes.c_double, dp, ctypes.c_int, ctypes.c_double, vp, vp,
                                           ctypes.POINTER(lqcd_solve_info)]),
        "lqcd_mscg_solve_dev": (ctypes.c_int, [vp, ctypes.c_double, dp, ctypes.c_int, ctypes.c_double, vp, vp,
                                               ctypes.POINTER(lqcd_solve_info), vp]),
        "lqcd_rational_apply": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_int,
                                               ctypes.c_double, vp, vp, dp, ctypes.POINTER(lqcd_solve_info)]),
        "lqcd_rational_apply_dev": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_int,
                                                   ctypes.c_double, vp, vp, dp, ctypes.POINTER(lqcd_solve_info),
                                                   vp]),
        "lqcd_cg_solve_mrhs": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                              ctypes.c_double, vp, vp, ctypes.POINTER(lqcd_solve_info)]),
        "lqcd_mscg_solve_packed": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, dp, ctypes.POINTER(dp), ip,
                                                  dp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                  ctypes.POINTER(lqcd_solve_info)]),
        "lqcd_profile_iteration": (ctypes.c_int, [vp, ctypes.c_double, dp, ctypes.c_int, ctypes.c_double, vp,
                                                  ctypes.c_int, dp, dp]),
        "lqcd_serve_create": (ctypes.c_int, [sz, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]),
        "lqcd_serve_register_field": (ctypes.c_int, [vp, ip, vp, sz, ip]),
        "lqcd_serve_submit": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double, dp, ctypes.c_int,
                                             ctypes.c_double, vp, ctypes.POINTER(ctypes.c_uint64)]),
        "lqcd_serve_poll": (ctypes.c_int, [vp, ctypes.c_uint64, vp, ctypes.POINTER(lqcd_solve_info)]),
        "lqcd_serve_drain": (ctypes.c_int, [vp, ctypes.c_double]),
        "lqcd_serve_stats_get": (ctypes.c_int, [vp, ctypes.POINTER(lqcd_serve_stats)]),
        "lqcd_serve_destroy": (None, [vp]),
        "lqcd_serve_set_opts": (ctypes.c_int, [vp, ctypes.POINTER(lqcd_opts)]),
        "lqcd_mom_upload": (ctypes.c_int, [vp, vp, sz]),
        "lqcd_mom_download": (ctypes.c_int, [vp, vp, sz]),
        "lqcd_gauge_mom_update": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
        "lqcd_gauge_link_update": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double]),
        "lqcd_gauge_md_steps": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]),
        "lqcd_gauge_action": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double, dp]),
        "lqcd_mom_energy": (ctypes.c_int, [vp, ctypes.c_int, dp]),
        "lqcd_fermion_force_update": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_int,
                                                     ctypes.c_double, vp, ctypes.c_double, dp,
                                                     ctypes.POINTER(lqcd_solve_info)]),
        "lqcd_deo_apply_mrhs_layout": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                      vp, vp, vp]),
        "lqcd_selftest_stage_wait": (ctypes.c_int, [vp, ctypes.c_double]),
        "lqcd_inject_alloc_failure": (None, [ctypes.c_long]),
        "lqcd_bounds_errors": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint)]),
        "lqcd_stout_smear": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_int]),
        "lqcd_stout_restore": (ctypes.c_int, [vp]),
        "lqcd_stout_force": (ctypes.c_int, [vp, vp, vp, ctypes.c_size_t]),
        "lqcd_deo_tuned_config": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ip]),
        "lqcd_measure_fma_rates": (ctypes.c_int, [dp, dp]),
        "lqcd_deo_apply_h16": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, vp, vp, vp]),
        "lqcd_shard_create": (ctypes.c_int, [ip, ctypes.c_int, ctypes.c_int, ctypes.POINTER(lqcd_opts),
                                             ctypes.POINTER(vp)]),
        "lqcd_shard_geometry": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_long)]),
        "lqcd_shard_links_upload": (ctypes.c_int, [vp, vp, sz]),
        "lqcd_shard_deo_apply": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, vp]),
        "lqcd_shard_exchange": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)]),
        "lqcd_shard_cg_solve": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, vp, vp, ctypes.POINTER(lqcd_solve_info)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(status: int) -> int:
    if status not in (LQCD_OK,):
        msg = _lib.lqcd_last_error().decode() if _lib else ""
        raise LqcdError(status, msg)
    return status


def default_opts(**kw) -> lqcd_opts:
    o = lqcd_opts()
    load().lqcd_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _c128(a, shape) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.reshape(shape)


def _dptr(t) -> int:
    """Device pointer of a contiguous CUDA torch tensor."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device arguments must be contiguous CUDA tensors")
    return t.data_ptr()


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream))


def to_device_spinor(a: np.ndarray, dtype=None, device="cuda"):
    """Canonical host [..., Vh, 3] -> device structure of arrays [..., 3, Vh]."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(np.swapaxes(a, -1, -2)))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device).contiguous()


def to_device_h16(a: np.ndarray, device="cuda"):
    """Canonical host [Vh, 3] -> (halves float16 [3, Vh, 2], norms float32 [Vh]):
    the per-site norm is the largest |re|, |im| of the site (1 for a zero
    site), the halves the values over it, rounded to FP16."""
    import torch
    a = np.asarray(a, np.complex128)
    m = np.maximum(np.abs(a.real), np.abs(a.imag)).max(axis=1)
    m = np.where(m > 0, m, 1.0)
    s = a / m[:, None]
    h = np.stack([s.real, s.imag], axis=-1).transpose(1, 0, 2)       # [3, Vh, 2]
    return (torch.from_numpy(np.ascontiguousarray(h)).to(torch.float16).to(device),
            torch.from_numpy(m.astype(np.float32)).to(device))


def from_device_h16(h, norm) -> np.ndarray:
    """(halves [3, Vh, 2], norms [Vh]) -> canonical host [Vh, 3] complex128."""
    hv = h.detach().float().cpu().numpy().astype(np.float64)
    nv = norm.detach().cpu().numpy().astype(np.float64)
    z = (hv[..., 0] + 1j * hv[..., 1]) * nv[None, :]
    return np.ascontiguousarray(z.T)


def from_device_spinor(t) -> np.ndarray:
    """Device [..., 3, Vh] -> canonical host [..., Vh, 3] complex128."""
    a = t.detach().cpu().numpy()
    return np.ascontiguousarray(np.swapaxes(a, -1, -2)).astype(np.complex128)


class Context:
    """One lattice on the current CUDA device (wraps lqcd_ctx)."""

    def __init__(self, dims, opts: lqcd_opts | None = None, **kw):
        self.lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.Vh = self.V // 2
        o = opts if opts is not None else default_opts(**kw)
        h = ctypes.c_void_p()
        check(self.lib.lqcd_create((ctypes.c_int * 4)(*self.dims), ctypes.byref(o), ctypes.byref(h)))
        self.h = h
        self.opts = o

    def close(self):
        if getattr(self, "h", None):
            self.lib.lqcd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_opts(self, **kw):
        for k, v in kw.items():
            setattr(self.opts, k, v)
        check(self.lib.lqcd_set_opts(self.h, ctypes.byref(self.opts)))

    def device_bytes(self) -> int:
        return int(self.lib.lqcd_device_bytes(self.h))

    # ------------------------------------------------------------- links
    def links_upload(self, links: np.ndarray):
        u = _c128(links, (4, self.V, 3, 3))
        check(self.lib.lqcd_links_upload(self.h, _ptr(u), u.size * 2))

    def links_download(self) -> np.ndarray:
        u = np.empty((4, self.V, 3, 3), np.complex128)
        check(self.lib.lqcd_links_download(self.h, _ptr(u), u.size * 2))
        return u

    # ------------------------------------------------- gauge molecular dynamics
    def mom_upload(self, H: np.ndarray):
        h = _c128(H, (4, self.V, 3, 3))
        check(self.lib.lqcd_mom_upload(self.h, _ptr(h), h.size * 2))

    def mom_download(self) -> np.ndarray:
        h = np.empty((4, self.V, 3, 3), np.complex128)
        check(self.lib.lqcd_mom_download(self.h, _ptr(h), h.size * 2))
        return h

    def gauge_mom_update(self, beta: float, eps: float, prec: int = 0):
        check(self.lib.lqcd_gauge_mom_update(self.h, int(prec), float(beta), float(eps)))

    def gauge_link_update(self, eps: float, prec: int = 0):
        check(self.lib.lqcd_gauge_link_update(self.h, int(prec), float(eps)))

    def gauge_md_steps(self, beta: float, eps: float, n_steps: int = 1, prec: int = 0):
        check(self.lib.lqcd_gauge_md_steps(self.h, int(prec), float(beta), float(eps), int(n_steps)))

    def gauge_action(self, beta: float, prec: int = 0) -> float:
        s = ctypes.c_double()
        check(self.lib.lqcd_gauge_action(self.h, int(prec), float(beta), ctypes.byref(s)))
        return s.value

    def fermion_force_update(self, mass: float, a0: float, a, shifts, tol: float, phi: np.ndarray, eps: float):
        """H <- H - eps F_f for S_f = phi^dag r(A) phi; returns (S_f, info)."""
        aa = np.ascontiguousarray(a, dtype=np.float64)
        sh = np.ascontiguousarray(shifts, dtype=np.float64)
        if aa.size != sh.size:
            raise ValueError("one coefficient per pole")
        pp = _c128(phi, (self.Vh, 3))
        act = ctypes.c_double()
        info = lqcd_solve_info()
        dp = ctypes.POINTER(ctypes.c_double)
        check(self.lib.lqcd_fermion_force_update(self.h, float(mass), float(a0), aa.ctypes.data_as(dp),
                                                 sh.ctypes.data_as(dp), sh.size, float(tol), _ptr(pp), float(eps),
                                                 ctypes.byref(act), ctypes.byref(info)))
        return act.value, info.as_dict()

    def selftest_stage_wait(self, limit_s: float = 0.05):
        """Run the bounded-wait self-test (lqcd_selftest_stage_wait); raises
        LqcdError with status LQCD_ETIMEOUT when the wait ran out as designed."""
        check(self.lib.lqcd_selftest_stage_wait(self.h, float(limit_s)))

    def stout_smear(self, rho: float, levels: int):
        """Smear the links `levels` times (lqcd_stout_smear)."""
        check(self.lib.lqcd_stout_smear(self.h, float(rho), int(levels)))

    def stout_restore(self):
        """Put the unsmeared links back (lqcd_stout_restore)."""
        check(self.lib.lqcd_stout_restore(self.h))

    def stout_force(self, F_smeared) -> np.ndarray:
        """Force on the thin links from one on the smeared links, [4][V][3][3]."""
        Fs = _c128(F_smeared, (4, self.V, 3, 3))
        out = np.empty_like(Fs)
        check(self.lib.lqcd_stout_force(self.h, _ptr(Fs), _ptr(out), Fs.size * 2))
        return out

    def mom_energy(self, prec: int = 0) -> float:
        k = ctypes.c_double()
        check(self.lib.lqcd_mom_energy(self.h, int(prec), ctypes.byref(k)))
        return k.value

    # --------------------------------------------------------------- D_eo
    def deo_apply(self, out_parity: int, inp: np.ndarray) -> np.ndarray:
        """Host call: canonical [Vh, 3] complex128 in and out."""
        a = _c128(inp, (self.Vh, 3))
        out = np.empty_like(a)
        check(self.lib.lqcd_deo_apply(self.h, int(out_parity), _ptr(a), _ptr(out), 0, None))
        return out

    def deo_apply_host_noalloc(self, out_parity: int, inp: np.ndarray) -> np.ndarray:
        """Host call staged through the library's fixed device array (no device
        allocation; lattices with V/2 <= 131072 sites)."""
        a = _c128(inp, (self.Vh, 3))
        out = np.empty_like(a)
        check(self.lib.lqcd_deo_apply_host_noalloc(self.h, int(out_parity), _ptr(a), _ptr(out)))
        return out

    def deo_apply_dev(self, out_parity: int, inp, out, stream=None):
        """Device call (FP64): complex128 [3, Vh] tensors."""
        check(self.lib.lqcd_deo_apply(self.h, int(out_parity), _dptr(inp), _dptr(out), 1, _stream_ptr(stream)))

    def deo_apply_ex(self, out_parity: int, prec: int, recon: int, inp, out, stream=None):
        check(self.lib.lqcd_deo_apply_ex(self.h, int(out_parity), int(prec), int(recon), _dptr(inp), _dptr(out),
                                         _stream_ptr(stream)))

    def deo_apply_h16(self, out_parity: int, h_in, n_in, h_out, n_out, stream=None):
        """D_eo with FP16 links and FP16 spinors with per-site norms (device)."""
        check(self.lib.lqcd_deo_apply_h16(self.h, int(out_parity), _dptr(h_in), _dptr(n_in), _dptr(h_out),
                                          _dptr(n_out), _stream_ptr(stream)))

    def deo_tuned_config(self, prec: int, recon: int) -> int:
        """The autotuner's launch code for deo_apply_ex(prec, recon) (0: not tuned yet)."""
        code = ctypes.c_int()
        check(self.lib.lqcd_deo_tuned_config(self.h, int(prec), int(recon), ctypes.byref(code)))
        return code.value

    def deo_apply_mrhs(self, out_parity: int, n_rhs: int, recon: int, inp, out, stream=None, layout: int = 0):
        """Multi-RHS D on device batches: layout 0 [3][Vh][n], 1 [3][n][Vh]."""
        if layout == 0:
            check(self.lib.lqcd_deo_apply_mrhs(self.h, int(out_parity), int(n_rhs), int(recon), _dptr(inp),
                                               _dptr(out), _stream_ptr(stream)))
        else:
            check(self.lib.lqcd_deo_apply_mrhs_layout(self.h, int(out_parity), int(n_rhs), int(recon), int(layout),
                                                      _dptr(inp), _dptr(out), _stream_ptr(stream)))

    # ------------------------------------------------------------- solvers
    def mscg_solve(self, mass: float, shifts, tol: float, b: np.ndarray, allow_noconv: bool = False,
                   out: np.ndarray | None = None):
        """Host call: returns (x [n_shift, Vh, 3], info dict).  `out`, a
        C-contiguous complex128 array of that shape, receives x instead of a
        new array (a reused buffer avoids first-touch page faults)."""
        sh = np.ascontiguousarray(shifts, dtype=np.float64)
        bb = _c128(b, (self.Vh, 3))
        shape = (sh.size, self.Vh, 3)
        if out is None:
            x = np.empty(shape, np.complex128)
        else:
            if out.shape != shape or out.dtype != np.complex128 or not out.flags.c_contiguous:
                raise ValueError(f"out must be a C-contiguous complex128 array of shape {shape}")
            x = out
        info = lqcd_solve_info()
        st = self.lib.lqcd_mscg_solve(self.h, float(mass), sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      sh.size, float(tol), _ptr(bb), _ptr(x), ctypes.byref(info))
        if not (allow_noconv and st == LQCD_ENOCONV):
            check(st)
        return x, info.as_dict()

    def rational_apply(self, mass: float, a0: float, a, shifts, tol: float, b: np.ndarray,
                       allow_noconv: bool = False):
        """Host call: y = a0 b + sum_i a_i (A + shifts_i)^{-1} b; returns (y [Vh, 3], Re <b, y>, info)."""
        aa = np.ascontiguousarray(a, dtype=np.float64)
        sh = np.ascontiguousarray(shifts, dtype=np.float64)
        if aa.size != sh.size:
            raise ValueError("one coefficient per pole")
        bb = _c128(b, (self.Vh, 3))
        y = np.empty_like(bb)
        act = ctypes.c_double()
        info = lqcd_solve_info()
        dp = ctypes.POINTER(ctypes.c_double)
        st = self.lib.lqcd_rational_apply(self.h, float(mass), float(a0), aa.ctypes.data_as(dp),
                                          sh.ctypes.data_as(dp), sh.size, float(tol), _ptr(bb), _ptr(y),
                                          ctypes.byref(act), ctypes.byref(info))
        if not (allow_noconv and st == LQCD_ENOCONV):
            check(st)
        return y, act.value, info.as_dict()

    def rational_apply_dev(self, mass: float, a0: float, a, shifts, tol: float, b, y, stream=None):
        """Device call: b, y complex128 [3, Vh]; returns (Re <b, y>, info)."""
        aa = np.ascontiguousarray(a, dtype=np.float64)
        sh = np.ascontiguousarray(shifts, dtype=np.float64)
        if aa.size != sh.size:
            raise ValueError("one coefficient per pole")
        act = ctypes.c_double()
        info = lqcd_solve_info()
        dp = ctypes.POINTER(ctypes.c_double)
        check(self.lib.lqcd_rational_apply_dev(self.h, float(mass), float(a0), aa.ctypes.data_as(dp),
                                               sh.ctypes.data_as(dp), sh.size, float(tol), _dptr(b), _dptr(y),
                                               ctypes.byref(act), ctypes.byref(info), _stream_ptr(stream)))
        return act.value, info.as_dict()

    def mscg_solve_dev(self, mass: float, shifts, tol: float, b, x, stream=None, allow_noconv=False):
        """Device call: b complex128 [3, Vh], x complex128 [n_shift, 3, Vh]."""
        sh = np.ascontiguousarray(shifts, dtype=np.float64)
        info = lqcd_solve_info()
        st = self.lib.lqcd_mscg_solve_dev(self.h, float(mass), sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          sh.size, float(tol), _dptr(b), _dptr(x), ctypes.byref(info),
                                          _stream_ptr(stream))
        if not (allow_noconv and st == LQCD_ENOCONV):
            check(st)
        return info.as_dict()

    def profile_iteration(self, mass: float, shifts, b, tol: float = 1e-10, iters: int = 20):
        """Per-kernel average ms of one solver iteration (see lqcd_profile_iteration)."""
        sh = np.ascontiguousarray(shifts, dtype=np.float64)
        ms = (ctypes.c_double * 4)()
        nact = ctypes.c_double()
        check(self.lib.lqcd_profile_iteration(self.h, float(mass), sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                              sh.size, float(tol), _dptr(b), int(iters), ms, ctypes.byref(nact)))
        return list(ms), nact.value

    def cg_solve_mrhs(self, mass: float, sigma: float, tol: float, b: np.ndarray):
        """Host call: b [n_rhs, Vh, 3]; returns (x, [info per rhs])."""
        bb = np.ascontiguousarray(b, dtype=np.complex128)
        n = bb.shape[0]
        x = np.empty_like(bb)
        infos = (lqcd_solve_info * n)()
        check(self.lib.lqcd_cg_solve_mrhs(self.h, float(mass), float(sigma), n, float(tol), _ptr(bb), _ptr(x),
                                          infos))
        return x, [i.as_dict() for i in infos]


def mscg_solve_packed(ctxs, masses, shifts_list, tols, bs):
    """One multi-shift solve per context, all advanced in shared launches."""
    lib = load()
    n = len(ctxs)
    hs = (ctypes.c_void_p * n)(*[c.h for c in ctxs])
    ms = (ctypes.c_double * n)(*[float(m) for m in masses])
    sh_arr = [np.ascontiguousarray(s, dtype=np.float64) for s in shifts_list]
    shp = (ctypes.POINTER(ctypes.c_double) * n)(*[a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in sh_arr])
    ns = (ctypes.c_int * n)(*[a.size for a in sh_arr])
    ts = (ctypes.c_double * n)(*[float(t) for t in tols])
    b_arr = [_c128(b, (c.Vh, 3)) for c, b in zip(ctxs, bs)]
    x_arr = [np.empty((a.size, c.Vh, 3), np.complex128) for a, c in zip(sh_arr, ctxs)]
    bp = (ctypes.c_void_p * n)(*[_ptr(a) for a in b_arr])
    xp = (ctypes.c_void_p * n)(*[_ptr(a) for a in x_arr])
    infos = (lqcd_solve_info * n)()
    check(lib.lqcd_mscg_solve_packed(hs, n, ms, shp, ns, ts, bp, xp, infos))
    return x_arr, [i.as_dict() for i in infos]


class ShardWorld:
    """All ranks of a t-slab decomposition of one lattice in this process,
    one shard context per rank (wraps lqcd_shard_*)."""

    def __init__(self, dims, world: int, opts: lqcd_opts | None = None, **kw):
        self.lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.world = int(world)
        self.Vh = int(np.prod(self.dims)) // 2
        o = opts if opts is not None else default_opts(**kw)
        self.h = []
        for r in range(self.world):
            h = ctypes.c_void_p()
            st = self.lib.lqcd_shard_create((ctypes.c_int * 4)(*self.dims), self.world, r, ctypes.byref(o),
                                            ctypes.byref(h))
            if st != LQCD_OK:
                self.close()
                check(st)
            self.h.append(h)
        info = (ctypes.c_long * 6)()
        check(self.lib.lqcd_shard_geometry(self.h[0], info))
        self.t0_step, self.nt, self.vh_ext, self.face, self.lo, self.hi = (int(v) for v in info)

    def close(self):
        for h in getattr(self, "h", []):
            if h:
                self.lib.lqcd_destroy(h)
        self.h = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def links_upload(self, links: np.ndarray):
        a = _c128(links, (4, self.Vh * 2, 3, 3))
        for h in self.h:
            check(self.lib.lqcd_shard_links_upload(h, _ptr(a), a.size * 2))

    def scatter(self, field: np.ndarray, device="cuda"):
        """Global canonical half field [Vh, 3] -> per-rank device spinors of
        the extended slabs (owned slices filled, ghost slices zero)."""
        import torch
        out = []
        for r in range(self.world):
            ext = np.zeros((self.vh_ext, 3), np.complex128)
            ext[self.lo:self.hi] = field[r * (self.hi - self.lo):(r + 1) * (self.hi - self.lo)]
            out.append(to_device_spinor(ext, device=device))
        torch.cuda.synchronize()
        return out

    def gather(self, fields) -> np.ndarray:
        """Owned slices of the per-rank device spinors -> global [Vh, 3]."""
        return np.concatenate([from_device_spinor(f)[self.lo:self.hi] for f in fields])

    def exchange(self, fields):
        hs = (ctypes.c_void_p * self.world)(*self.h)
        fp = (ctypes.c_void_p * self.world)(*[_dptr(f) for f in fields])
        check(self.lib.lqcd_shard_exchange(hs, self.world, fp))

    def deo_apply(self, out_parity: int, fields_in, fields_out):
        for h, a, b in zip(self.h, fields_in, fields_out):
            check(self.lib.lqcd_shard_deo_apply(h, int(out_parity), _dptr(a), _dptr(b), None))

    def cg_solve(self, mass: float, sigma: float, tol: float, b: np.ndarray):
        bb = _c128(b, (self.Vh, 3))
        x = np.zeros_like(bb)
        info = lqcd_solve_info()
        hs = (ctypes.c_void_p * self.world)(*self.h)
        check(self.lib.lqcd_shard_cg_solve(hs, self.world, float(mass), float(sigma), float(tol), _ptr(bb),
                                           _ptr(x), ctypes.byref(info)))
        return x, info.as_dict()


class Server:
    """Continuous-batching solve server (wraps lqcd_server)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 16, max_queue: int = 1024):
        self.lib = load()
        h = ctypes.c_void_p()
        check(self.lib.lqcd_serve_create(int(hbm_budget_bytes), int(max_slots), int(max_queue), ctypes.byref(h)))
        self.h = h
        self.fields = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.lqcd_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_opts(self, **kw):
        """Options of later requests (prec 0 = FP64, 1 = FP32 mixed; recon, fp64_until, ...)."""
        o = default_opts(**kw)
        check(self.lib.lqcd_serve_set_opts(self.h, ctypes.byref(o)))

    def register_field(self, dims, links: np.ndarray) -> int:
        dims = tuple(int(d) for d in dims)
        V = int(np.prod(dims))
        u = _c128(links, (4, V, 3, 3))
        fid = ctypes.c_int()
        check(self.lib.lqcd_serve_register_field(self.h, (ctypes.c_int * 4)(*dims), _ptr(u), u.size * 2,
                                                 ctypes.byref(fid)))
        self.fields[fid.value] = dims
        return fid.value

    def submit(self, field_id: int, mass: float, shifts, tol: float, b: np.ndarray) -> int:
        """Returns a ticket; raises LqcdError(LQCD_EBUSY / LQCD_ENOMEM) on rejection."""
        sh = np.ascontiguousarray(shifts, dtype=np.float64)
        dims = self.fields.get(field_id)
        bb = _c128(b, (int(np.prod(dims)) // 2, 3) if dims else np.shape(b))
        t = ctypes.c_uint64()
        check(self.lib.lqcd_serve_submit(self.h, int(field_id), float(mass),
                                         sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), sh.size, float(tol),
                                         _ptr(bb), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, field_id: int, n_shift: int):
        """(x, info) when finished, None while running."""
        V = int(np.prod(self.fields[field_id]))
        x = np.empty((n_shift, V // 2, 3), np.complex128)
        info = lqcd_solve_info()
        st = self.lib.lqcd_serve_poll(self.h, ctypes.c_uint64(ticket), _ptr(x), ctypes.byref(info))
        if st == LQCD_ENOTREADY:
            return None
        check(st)
        return x, info.as_dict()

    def drain(self, timeout_s: float = 0.0):
        check(self.lib.lqcd_serve_drain(self.h, float(timeout_s)))

    def stats(self) -> dict:
        st = lqcd_serve_stats()
        check(self.lib.lqcd_serve_stats_get(self.h, ctypes.byref(st)))
        return st.as_dict()


def measure_fma_rates() -> dict:
    """FP64 and FP32 FMA issue rates of the current device (FMA per second)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    check(load().lqcd_measure_fma_rates(ctypes.byref(a), ctypes.byref(b)))
    return {"fp64_fma_per_s": a.value, "fp32_fma_per_s": b.value}


def inject_alloc_failure(k: int):
    """The k-th device allocation from now fails with LQCD_ENOMEM (k <= 0
    disarms); see lqcd_inject_alloc_failure."""
    load().lqcd_inject_alloc_failure(int(k))


def bounds_errors() -> int:
    """Error bits recorded by a bounds-checked library since the last call
    (lqcd_bounds_errors); LqcdError(LQCD_ESTATE) for the default build."""
    w = ctypes.c_uint()
    check(load().lqcd_bounds_errors(ctypes.byref(w)))
    return w.value
