"""ctypes front end of the plain C FP64 oracle (``lqcd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use this module; the product library never does.
It imports nothing from the CUDA package.

Every function mirrors one function of the C file, which cites the paper's
definitions (Eqs. lexicographic_eo, diracblock, lineqeo, shlineq).  Arrays are
numpy complex128 in the canonical host layouts:

* links  ``[4][V][3][3]``: U_mu(x)[row][col] at lexicographic index
  ``x0 + N0 (x1 + N1 (x2 + N2 x3))``;
* half-lattice fields ``[Vh][3]`` in the paper's ``idxh`` order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lqcd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs: dict[int, ctypes.CDLL] = {}


def so_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction, no -march)."""
    out = so_path(mutant)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = f"{out}.{os.getpid()}.tmp"
    cmd = ["gcc", "-std=gnu99", "-O2", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", f"-DORACLE_MUTANT={mutant}", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True)
    os.replace(tmp, out)
    return out


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    ip = ctypes.POINTER(ctypes.c_int)
    vp = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_lex.argtypes = [ip, ip]
    lib.oracle_lex.restype = ctypes.c_long
    lib.oracle_idxh.argtypes = [ip, ip]
    lib.oracle_idxh.restype = ctypes.c_long
    lib.oracle_parity.argtypes = [ip]
    lib.oracle_parity.restype = ctypes.c_int
    lib.oracle_link_sign.argtypes = [ip, ip, ctypes.c_int]
    lib.oracle_link_sign.restype = ctypes.c_double
    lib.oracle_deo.argtypes = [ip, ctypes.c_int, vp, vp, vp]
    lib.oracle_deo.restype = None
    lib.oracle_apply_A.argtypes = [ip, vp, ctypes.c_double, ctypes.c_double, vp, vp, vp]
    lib.oracle_apply_A.restype = None
    lib.oracle_true_residual.argtypes = [ip, vp, ctypes.c_double, ctypes.c_double, vp, vp]
    lib.oracle_true_residual.restype = ctypes.c_double
    lib.oracle_cg.argtypes = [ip, vp, ctypes.c_double, ctypes.c_double, vp, vp,
                              ctypes.c_double, ctypes.c_int]
    lib.oracle_cg.restype = ctypes.c_int
    lib.oracle_mscg.argtypes = [ip, vp, ctypes.c_double, dp, ctypes.c_int, vp, vp,
                                ctypes.c_double, ctypes.c_int, ip, ip, dp]
    lib.oracle_mscg.restype = ctypes.c_int
    lib.oracle_rational_apply.argtypes = [ip, vp, ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_int,
                                          vp, vp, ctypes.c_double, ctypes.c_int, dp]
    lib.oracle_rational_apply.restype = ctypes.c_int
    lib.oracle_fermion_force.argtypes = [ip, vp, ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_int, vp,
                                         ctypes.c_double, ctypes.c_int, vp, dp]
    lib.oracle_fermion_force.restype = ctypes.c_int
    lib.oracle_gauge_action.argtypes = [ip, vp, ctypes.c_double]
    lib.oracle_gauge_action.restype = ctypes.c_double
    lib.oracle_gauge_force.argtypes = [ip, vp, ctypes.c_double, vp]
    lib.oracle_gauge_force.restype = None
    lib.oracle_exp_iH.argtypes = [vp, ctypes.c_double, vp]
    lib.oracle_exp_iH.restype = None
    lib.oracle_mom_update.argtypes = [ip, vp, vp, ctypes.c_double, ctypes.c_double]
    lib.oracle_mom_update.restype = None
    lib.oracle_link_update.argtypes = [ip, vp, vp, ctypes.c_double]
    lib.oracle_link_update.restype = None
    lib.oracle_mom_energy.argtypes = [ip, vp]
    lib.oracle_mom_energy.restype = ctypes.c_double
    lib.oracle_stout_smear.argtypes = [ip, vp, ctypes.c_double, vp]
    lib.oracle_stout_smear.restype = None
    lib.oracle_stout_force.argtypes = [ip, vp, ctypes.c_double, vp, vp]
    lib.oracle_stout_force.restype = None
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_threads.restype = ctypes.c_int
    lib.oracle_mutant.restype = ctypes.c_int
    return lib


def load(mutant: int = 0) -> ctypes.CDLL:
    with _lock:
        if mutant not in _libs:
            _libs[mutant] = _bind(ctypes.CDLL(build(mutant)))
        return _libs[mutant]


class Oracle:
    """Typed wrapper around one build (default or a planted mutant)."""

    def __init__(self, mutant: int = 0):
        self.lib = load(mutant)
        self.mutant = mutant

    # ---------------------------------------------------------------- helpers
    @staticmethod
    def _dims(dims) -> ctypes.Array:
        d = [int(v) for v in dims]
        if len(d) != 4 or any(v < 2 or v % 2 for v in d):
            raise ValueError(f"lattice sides must be 4 even integers >= 2, got {dims}")
        return (ctypes.c_int * 4)(*d)

    @staticmethod
    def _c128(a, shape) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.complex128)
        if a.shape != tuple(shape):
            a = a.reshape(shape)
        return a

    @staticmethod
    def _ptr(a: np.ndarray) -> int:
        return a.ctypes.data

    # --------------------------------------------------------------- geometry
    def lex(self, dims, x) -> int:
        return self.lib.oracle_lex(self._dims(dims), (ctypes.c_int * 4)(*x))

    def idxh(self, dims, x) -> int:
        return self.lib.oracle_idxh(self._dims(dims), (ctypes.c_int * 4)(*x))

    def parity(self, x) -> int:
        return self.lib.oracle_parity((ctypes.c_int * 4)(*x))

    def link_sign(self, dims, x, mu) -> float:
        return self.lib.oracle_link_sign(self._dims(dims), (ctypes.c_int * 4)(*x), mu)

    # ---------------------------------------------------------------- operators
    def deo(self, dims, out_parity: int, links, inp) -> np.ndarray:
        """D_eo (out_parity 0: odd -> even) or D_oe (out_parity 1: even -> odd)."""
        V = int(np.prod(dims))
        links = self._c128(links, (4, V, 3, 3))
        inp = self._c128(inp, (V // 2, 3))
        out = np.empty((V // 2, 3), np.complex128)
        self.lib.oracle_deo(self._dims(dims), int(out_parity), self._ptr(links),
                            self._ptr(inp), self._ptr(out))
        return out

    def apply_A(self, dims, links, mass: float, sigma: float, inp) -> np.ndarray:
        """(m^2 + sigma) in - D_eo D_oe in on even sites."""
        V = int(np.prod(dims))
        links = self._c128(links, (4, V, 3, 3))
        inp = self._c128(inp, (V // 2, 3))
        out = np.empty_like(inp)
        tmp = np.empty_like(inp)
        self.lib.oracle_apply_A(self._dims(dims), self._ptr(links), float(mass),
                                float(sigma), self._ptr(inp), self._ptr(out), self._ptr(tmp))
        return out

    def true_residual(self, dims, links, mass, sigma, b, x) -> float:
        V = int(np.prod(dims))
        links = self._c128(links, (4, V, 3, 3))
        b = self._c128(b, (V // 2, 3))
        x = self._c128(x, (V // 2, 3))
        return self.lib.oracle_true_residual(self._dims(dims), self._ptr(links), float(mass),
                                             float(sigma), self._ptr(b), self._ptr(x))

    def cg(self, dims, links, mass, sigma, b, tol, max_iter=20000, x0=None):
        V = int(np.prod(dims))
        links = self._c128(links, (4, V, 3, 3))
        b = self._c128(b, (V // 2, 3))
        x = np.zeros_like(b) if x0 is None else np.array(x0, np.complex128).reshape(b.shape)
        it = self.lib.oracle_cg(self._dims(dims), self._ptr(links), float(mass), float(sigma),
                                self._ptr(b), self._ptr(x), float(tol), int(max_iter))
        return x, it

    def mscg(self, dims, links, mass, shifts, b, tol, max_iter=20000):
        """Returns (x [n_shift][Vh][3], info dict)."""
        V = int(np.prod(dims))
        links = self._c128(links, (4, V, 3, 3))
        b = self._c128(b, (V // 2, 3))
        sh = np.ascontiguousarray(shifts, dtype=np.float64)
        n = sh.size
        x = np.zeros((n, V // 2, 3), np.complex128)
        iters = (ctypes.c_int * 2)()
        shift_iters = (ctypes.c_int * max(n, 1))()
        resid = np.zeros(max(n, 1), np.float64)
        st = self.lib.oracle_mscg(self._dims(dims), self._ptr(links), float(mass),
                                  sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n,
                                  self._ptr(b), self._ptr(x), float(tol), int(max_iter),
                                  iters, shift_iters,
                                  resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        info = {"status": st, "iters": iters[0], "refine_iters": iters[1],
                "shift_iters": list(shift_iters)[:n], "true_resid": resid[:n].copy()}
        return x, info

    def rational_apply(self, dims, links, mass, a0, a, shifts, b, tol, max_iter=20000):
        """y = a0 b + sum_i a_i (A + shifts_i)^{-1} b and Re <b, y>; returns (y, action, status)."""
        V = int(np.prod(dims))
        links = self._c128(links, (4, V, 3, 3))
        b = self._c128(b, (V // 2, 3))
        aa = np.ascontiguousarray(a, dtype=np.float64)
        sh = np.ascontiguousarray(shifts, dtype=np.float64)
        if aa.size != sh.size:
            raise ValueError("one coefficient per shift")
        y = np.empty_like(b)
        act = ctypes.c_double()
        dp = ctypes.POINTER(ctypes.c_double)
        st = self.lib.oracle_rational_apply(self._dims(dims), self._ptr(links), float(mass), float(a0),
                                            aa.ctypes.data_as(dp), sh.ctypes.data_as(dp), sh.size,
                                            self._ptr(b), self._ptr(y), float(tol), int(max_iter),
                                            ctypes.byref(act))
        return y, act.value, st

    def fermion_force(self, dims, links, mass, a0, a, shifts, phi, tol, max_iter=20000):
        """Force of S_f = phi^dag r(A) phi on every link; returns (F [4][V][3][3], S_f, status)."""
        V = int(np.prod(dims))
        links = self._c128(links, (4, V, 3, 3))
        phi = self._c128(phi, (V // 2, 3))
        aa = np.ascontiguousarray(a, dtype=np.float64)
        sh = np.ascontiguousarray(shifts, dtype=np.float64)
        F = np.empty_like(links)
        act = ctypes.c_double()
        dp = ctypes.POINTER(ctypes.c_double)
        st = self.lib.oracle_fermion_force(self._dims(dims), self._ptr(links), float(mass), float(a0),
                                           aa.ctypes.data_as(dp), sh.ctypes.data_as(dp), sh.size, self._ptr(phi),
                                           float(tol), int(max_iter), self._ptr(F), ctypes.byref(act))
        return F, act.value, st

    # ------------------------------------------------- gauge MD (Symanzik)
    def gauge_action(self, dims, links, beta: float) -> float:
        V = int(np.prod(dims))
        links = self._c128(links, (4, V, 3, 3))
        return self.lib.oracle_gauge_action(self._dims(dims), self._ptr(links), float(beta))

    def gauge_force(self, dims, links, beta: float) -> np.ndarray:
        V = int(np.prod(dims))
        links = self._c128(links, (4, V, 3, 3))
        F = np.empty_like(links)
        self.lib.oracle_gauge_force(self._dims(dims), self._ptr(links), float(beta), self._ptr(F))
        return F

    def exp_iH(self, H, t: float) -> np.ndarray:
        H = self._c128(H, (3, 3))
        E = np.empty_like(H)
        self.lib.oracle_exp_iH(self._ptr(H), float(t), self._ptr(E))
        return E

    def mom_update(self, dims, links, mom, beta: float, eps: float) -> np.ndarray:
        """H - eps F(U) (a new array)."""
        V = int(np.prod(dims))
        links = self._c128(links, (4, V, 3, 3))
        H = np.array(self._c128(mom, (4, V, 3, 3)), copy=True)
        self.lib.oracle_mom_update(self._dims(dims), self._ptr(links), self._ptr(H), float(beta), float(eps))
        return H

    def link_update(self, dims, links, mom, eps: float) -> np.ndarray:
        """exp(i eps H) U for every link (a new array)."""
        V = int(np.prod(dims))
        U = np.array(self._c128(links, (4, V, 3, 3)), copy=True)
        H = self._c128(mom, (4, V, 3, 3))
        self.lib.oracle_link_update(self._dims(dims), self._ptr(U), self._ptr(H), float(eps))
        return U

    def mom_energy(self, dims, mom) -> float:
        V = int(np.prod(dims))
        H = self._c128(mom, (4, V, 3, 3))
        return self.lib.oracle_mom_energy(self._dims(dims), self._ptr(H))

    # ------------------------------------------------- stout smearing
    def stout_smear(self, dims, links, rho: float, levels: int = 1) -> np.ndarray:
        """U^(levels): the stout map applied `levels` times (a new array)."""
        return self.stout_levels(dims, links, rho, levels)[-1]

    def stout_levels(self, dims, links, rho: float, levels: int) -> list:
        """[U^(0) = U, U^(1), ..., U^(levels)]."""
        V = int(np.prod(dims))
        out = [np.array(self._c128(links, (4, V, 3, 3)), copy=True)]
        for _ in range(int(levels)):
            nxt = np.empty_like(out[-1])
            self.lib.oracle_stout_smear(self._dims(dims), self._ptr(out[-1]), float(rho), self._ptr(nxt))
            out.append(nxt)
        return out

    def stout_force(self, dims, links, rho: float, F_smeared, levels: int = 1) -> np.ndarray:
        """Force on the thin links U from the force on U^(levels), chained
        back one level at a time (oracle_stout_force)."""
        V = int(np.prod(dims))
        lv = self.stout_levels(dims, links, rho, levels)
        F = np.array(self._c128(F_smeared, (4, V, 3, 3)), copy=True)
        for k in range(int(levels) - 1, -1, -1):
            Fk = np.empty_like(F)
            self.lib.oracle_stout_force(self._dims(dims), self._ptr(lv[k]), float(rho), self._ptr(F), self._ptr(Fk))
            F = Fk
        return F

    def set_threads(self, n: int = 0) -> int:
        return self.lib.oracle_set_threads(int(n))


_default: Oracle | None = None


def oracle() -> Oracle:
    """The default (mutation-free) oracle build."""
    global _default
    if _default is None:
        _default = Oracle(0)
    return _default
