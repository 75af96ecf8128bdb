"""FP64 CPU oracle for the HQMC hot path (arXiv 2508.16298).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA library is checked against.  Only the test suite, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it; the library itself never
does, and nothing here imports the library.

The arithmetic lives in ``hqmc_oracle.c`` (double precision, matrix-free, in the
paper's order) and is reached through ctypes.  ``philox.py`` is a separate
counter-based generator written from its published definition, so that random
draws made on the GPU can be reproduced here bit for bit.

Array conventions: ``theta`` is float64 of shape (Ntau, L, L, 2) indexed
[tau, y, x, c] with c = 0 the bond (x,y)->(x+1,y) and c = 1 the bond
(x,y)->(x,y+1); vectors are complex128 of shape (Ntau, L, L) indexed [tau, y, x].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hqmc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libhqmc_oracle.so")

# -ffp-contract=off keeps the rounding identical on x86-64 and aarch64 hosts.
CFLAGS = ["-O3", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off"]


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/libhqmc_oracle.so`` (gcc)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Lat(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int),
        ("Ntau", ctypes.c_int),
        ("dtau", ctypes.c_double),
        ("t", ctypes.c_double),
        ("J", ctypes.c_double),
        ("K", ctypes.c_double),
        ("noncompact", ctypes.c_int),
    ]


@dataclass(frozen=True)
class Lattice:
    """Model and lattice parameters (Results, "Model"; Methods)."""

    L: int
    Ntau: int
    dtau: float = 0.1
    t: float = 1.0
    J: float = 1.0
    K: float = 0.0
    noncompact: bool = False

    @property
    def V(self) -> int:
        return self.L * self.L

    @property
    def n_sites(self) -> int:
        return self.V * self.Ntau

    def _c(self) -> _Lat:
        return _Lat(self.L, self.Ntau, self.dtau, self.t, self.J, self.K, int(self.noncompact))


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Lat)
        vp = ctypes.c_void_p
        d = ctypes.c_double
        i = ctypes.c_int
        ip = ctypes.POINTER(ctypes.c_int)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_apply_B.argtypes = [P, vp, vp, vp, i]
        lib.orc_apply_M.argtypes = [P, vp, vp, vp, i]
        lib.orc_apply_MdagM.argtypes = [P, vp, vp, vp]
        lib.orc_dot.argtypes = [ctypes.c_long, vp, vp, dp, dp]
        lib.orc_cg.argtypes = [P, vp, vp, vp, d, i, ip, dp]
        lib.orc_cg.restype = i
        lib.orc_fermion_dS.argtypes = [P, vp, vp, vp]
        lib.orc_bosonic_action.argtypes = [P, vp]
        lib.orc_bosonic_action.restype = d
        lib.orc_bosonic_dS.argtypes = [P, vp, vp]
        lib.orc_fermion_action.argtypes = [P, vp, vp]
        lib.orc_fermion_action.restype = d
        lib.orc_leapfrog.argtypes = [P, vp, vp, vp, vp, i, d, d, i, ip]
        lib.orc_leapfrog.restype = i
        lib.orc_trajectory.argtypes = [P, vp, vp, vp, d, i, d, d, i, dp, dp, ip, ip]
        lib.orc_trajectory.restype = i
        lib.orc_num_threads.restype = i
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _theta(lat: Lattice, theta) -> np.ndarray:
    a = np.ascontiguousarray(theta, dtype=np.float64)
    assert a.size == 2 * lat.n_sites, a.shape
    return a


def _vec(lat: Lattice, v) -> np.ndarray:
    a = np.ascontiguousarray(v, dtype=np.complex128)
    assert a.size == lat.n_sites, a.shape
    return a


def num_threads() -> int:
    return _load().orc_num_threads()


def apply_B(lat: Lattice, theta_slice, v, adjoint: bool = False) -> np.ndarray:
    """B v (or B^dagger v) for one slice, Eq. (eq24)."""
    th = np.ascontiguousarray(theta_slice, dtype=np.float64)
    vin = np.ascontiguousarray(v, dtype=np.complex128)
    assert th.size == 2 * lat.V and vin.size == lat.V
    out = np.empty_like(vin)
    _load().orc_apply_B(ctypes.byref(lat._c()), _ptr(th), _ptr(vin), _ptr(out), int(adjoint))
    return out


def apply_M(lat: Lattice, theta, x, dagger: bool = False) -> np.ndarray:
    """M x or M^dagger x, Eq. (M_alpha)."""
    th, xv = _theta(lat, theta), _vec(lat, x)
    y = np.empty_like(xv)
    _load().orc_apply_M(ctypes.byref(lat._c()), _ptr(th), _ptr(xv), _ptr(y), int(dagger))
    return y


def apply_MdagM(lat: Lattice, theta, x) -> np.ndarray:
    th, xv = _theta(lat, theta), _vec(lat, x)
    y = np.empty_like(xv)
    _load().orc_apply_MdagM(ctypes.byref(lat._c()), _ptr(th), _ptr(xv), _ptr(y))
    return y


def dot(a, b) -> complex:
    """<a, b> = sum conj(a) b in index order."""
    av = np.ascontiguousarray(a, dtype=np.complex128)
    bv = np.ascontiguousarray(b, dtype=np.complex128)
    re, im = ctypes.c_double(), ctypes.c_double()
    _load().orc_dot(av.size, _ptr(av), _ptr(bv), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def cg(lat: Lattice, theta, phi, x0=None, tol: float = 1e-10, maxit: int = 100000):
    """Solve (M^dagger M) X = phi, Eq. (pCG) with identity preconditioner.

    Returns (X, iterations, true_residual, status) with status 0 converged, 1 not."""
    th, ph = _theta(lat, theta), _vec(lat, phi)
    x = np.zeros_like(ph) if x0 is None else _vec(lat, x0).copy()
    it, res = ctypes.c_int(), ctypes.c_double()
    st = _load().orc_cg(ctypes.byref(lat._c()), _ptr(th), _ptr(ph), _ptr(x), tol, maxit,
                        ctypes.byref(it), ctypes.byref(res))
    return x, it.value, res.value, st


def fermion_dS(lat: Lattice, theta, X) -> np.ndarray:
    """d/dtheta [eta^dagger (M^dagger M)^{-1} eta] given X = (M^dagger M)^{-1} eta."""
    th, xv = _theta(lat, theta), _vec(lat, X)
    out = np.empty(th.shape, dtype=np.float64)
    _load().orc_fermion_dS(ctypes.byref(lat._c()), _ptr(th), _ptr(xv), _ptr(out))
    return out


def bosonic_action(lat: Lattice, theta) -> float:
    return _load().orc_bosonic_action(ctypes.byref(lat._c()), _ptr(_theta(lat, theta)))


def bosonic_dS(lat: Lattice, theta) -> np.ndarray:
    th = _theta(lat, theta)
    out = np.empty(th.shape, dtype=np.float64)
    _load().orc_bosonic_dS(ctypes.byref(lat._c()), _ptr(th), _ptr(out))
    return out


def fermion_action(lat: Lattice, eta, X) -> float:
    return _load().orc_fermion_action(ctypes.byref(lat._c()), _ptr(_vec(lat, eta)), _ptr(_vec(lat, X)))


def leapfrog(lat: Lattice, theta, p, eta, X0=None, nsteps: int = 10, dt: float = 0.02,
             tol: float = 1e-12, maxit: int = 100000):
    """Eq. (leapfrog).  Returns (theta, p, X, cg_iterations, unconverged_solves)."""
    th = _theta(lat, theta).copy()
    pv = np.ascontiguousarray(p, dtype=np.float64).copy()
    ev = _vec(lat, eta)
    X = np.zeros_like(ev) if X0 is None else _vec(lat, X0).copy()
    it = ctypes.c_int()
    bad = _load().orc_leapfrog(ctypes.byref(lat._c()), _ptr(th), _ptr(pv), _ptr(ev), _ptr(X),
                               nsteps, dt, tol, maxit, ctypes.byref(it))
    return th, pv, X, it.value, bad


def trajectory(lat: Lattice, theta, p0, R, u: float, nsteps: int = 10, dt: float = 0.02,
               tol: float = 1e-12, maxit: int = 100000) -> dict:
    """One HQMC update (Methods, steps (i)-(iv)) with supplied Gaussian draws."""
    th = _theta(lat, theta).copy()
    pv = np.ascontiguousarray(p0, dtype=np.float64)
    Rv = _vec(lat, R)
    H0, H1 = ctypes.c_double(), ctypes.c_double()
    acc, it = ctypes.c_int(), ctypes.c_int()
    bad = _load().orc_trajectory(ctypes.byref(lat._c()), _ptr(th), _ptr(pv), _ptr(Rv), u, nsteps,
                                 dt, tol, maxit, ctypes.byref(H0), ctypes.byref(H1),
                                 ctypes.byref(acc), ctypes.byref(it))
    return {"theta": th, "H0": H0.value, "H1": H1.value, "dH": H1.value - H0.value,
            "accepted": bool(acc.value), "cg_iterations": it.value, "unconverged": bad}
