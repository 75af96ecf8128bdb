"""ctypes binding of libhqmc (include/hqmc.h) for torch CUDA tensors.

Argument marshalling only: every step runs in the library's CUDA kernels.
PyTorch supplies device memory and the current stream.  Importing this module
loads ``libhqmc.so`` and raises ImportError if it has not been built; there is
no CPU fallback.

Shapes and dtypes (all CUDA, contiguous):
  theta, p, F : float64 (Ntau, L, L, 2)
  vectors     : complex128 (Ntau, L, L); complex64 selects the FP32 operators.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhqmc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2508_16298_gb300.build.build() "
                      "(needs the CUDA toolkit); there is no CPU fallback")
_lib = ctypes.CDLL(LIB_PATH)

OK, EINVAL, ENOTCONV, EBREAKDOWN, ENONFINITE, ETIMEOUT, ECUDA, ENOMEM, EUNSUPPORTED, EIO = range(10)
FP64, FP32 = 0, 1
ACTION_COMPACT, ACTION_NONCOMPACT = 0, 1
SOLVER_CG64, SOLVER_MIXED, SOLVER_LEARNED, SOLVER_PCG64, SOLVER_PMIXED, SOLVER_PLEARNED, SOLVER_FLEARNED = range(7)
SOLVERS = {"cg64": SOLVER_CG64, "mixed": SOLVER_MIXED, "learned": SOLVER_LEARNED, "pcg64": SOLVER_PCG64,
           "pmixed": SOLVER_PMIXED, "plearned": SOLVER_PLEARNED, "flearned": SOLVER_FLEARNED}
TIMER_MDAGM, TIMER_CG_UPDATE, TIMER_FORCE, TIMER_MDAGM32, TIMER_PRECOND = 0, 1, 2, 3, 4

# Every function declared in include/hqmc.h.
EXPORTS = ("hqmc_make_config", "hqmc_free_config", "hqmc_strerror", "hqmc_last_error", "hqmc_num_sites",
           "hqmc_launch_count", "hqmc_get_launch_shape",
           "hqmc_apply_M", "hqmc_apply_MdagM", "hqmc_apply_precond", "hqmc_get_precond", "hqmc_get_precond_shape",
           "hqmc_set_precond_fused", "hqmc_cg_solve",
           "hqmc_estimate", "hqmc_estimate_projected", "hqmc_set_multi_rhs", "hqmc_set_multi_ranges", "hqmc_multi_launch_shape",
           "hqmc_cg_solve_multi", "hqmc_estimate_multi",
           "hqmc_force", "hqmc_action_terms",
           "hqmc_draw", "hqmc_leapfrog", "hqmc_trajectory", "hqmc_set_timing", "hqmc_get_timing", "hqmc_get_timing_samples",
           "hqmc_probe_fp64_rate", "hqmc_apply_MdagM_static", "hqmc_make_batch", "hqmc_free_batch",
           "hqmc_batch_last_error", "hqmc_batch_launch_count", "hqmc_batch_cg_solve", "hqmc_batch_trajectory",
           "hqmc_batch_set_solver", "hqmc_batch_launch_shape",
           "hqmc_net_create", "hqmc_net_free", "hqmc_net_num_weights", "hqmc_net_get_weights",
           "hqmc_net_set_weights", "hqmc_net_apply", "hqmc_net_train_step", "hqmc_set_preconditioner",
           "hqmc_set_net_interval", "hqmc_set_net_tensor_cores", "hqmc_set_guess_history", "hqmc_checkpoint_write", "hqmc_checkpoint_read")


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("Ntau", ctypes.c_int), ("dtau", ctypes.c_double),
                ("t", ctypes.c_double), ("J", ctypes.c_double), ("K", ctypes.c_double),
                ("action", ctypes.c_int), ("reliable_interval", ctypes.c_int), ("autotune", ctypes.c_int),
                ("variant", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("reliable_updates", ctypes.c_int), ("true_residual", ctypes.c_double),
                ("recursive_residual", ctypes.c_double), ("fp64_fallback", ctypes.c_int),
                ("net_guess_used", ctypes.c_int), ("fcg_fallback", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class TrajInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("accepted", ctypes.c_int), ("cg_solves", ctypes.c_int),
                ("cg_iterations", ctypes.c_int), ("H0", ctypes.c_double), ("H1", ctypes.c_double),
                ("dH", ctypes.c_double), ("u", ctypes.c_double), ("max_true_residual", ctypes.c_double),
                ("net_guesses_tried", ctypes.c_int), ("net_guesses_used", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Checkpoint(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("Ntau", ctypes.c_int), ("dtau", ctypes.c_double), ("t", ctypes.c_double),
                ("J", ctypes.c_double), ("K", ctypes.c_double), ("action", ctypes.c_int), ("n_weights", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("traj_counter", ctypes.c_uint64), ("dt", ctypes.c_double),
                ("nsteps", ctypes.c_int), ("solver", ctypes.c_int), ("trajectories", ctypes.c_longlong),
                ("accepted", ctypes.c_longlong), ("version", ctypes.c_int), ("reserved", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp, _i, _d, _u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
_sig = {
    "hqmc_make_config": ([ctypes.POINTER(Params), ctypes.POINTER(_vp)], _i),
    "hqmc_free_config": ([_vp], _i),
    "hqmc_strerror": ([_i], ctypes.c_char_p),
    "hqmc_last_error": ([_vp], ctypes.c_char_p),
    "hqmc_num_sites": ([_vp], ctypes.c_longlong),
    "hqmc_launch_count": ([_vp], ctypes.c_longlong),
    "hqmc_get_launch_shape": ([_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                               ctypes.POINTER(ctypes.c_float)], _i),
    "hqmc_apply_M": ([_vp, _vp, _vp, _vp, _i, _i, _vp], _i),
    "hqmc_apply_MdagM": ([_vp, _vp, _vp, _vp, _i, _vp], _i),
    "hqmc_apply_precond": ([_vp, _vp, _vp, _i, _vp], _i),
    "hqmc_get_precond_shape": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                               ctypes.c_int),
    "hqmc_set_precond_fused": ([_vp, _i, _i], _i),
    "hqmc_get_precond": ([_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i)], _i),
    "hqmc_cg_solve": ([_vp, _vp, _vp, _vp, _d, _i, _i, ctypes.POINTER(SolveInfo), _vp], _i),
    "hqmc_estimate": ([_vp, _vp, ctypes.c_uint64, ctypes.c_uint64, _i, _d, _i, _i, _vp, _vp,
                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolveInfo), _vp], _i),
    "hqmc_estimate_projected": ([_vp, _vp, ctypes.c_uint64, ctypes.c_uint64, _i, _d, _i, _i, _vp, _vp,
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolveInfo), _vp], _i),
    "hqmc_set_multi_rhs": ([_vp, _i], _i),
    "hqmc_set_multi_ranges": ([_vp, _i], _i),
    "hqmc_multi_launch_shape": ([_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)], _i),
    "hqmc_cg_solve_multi": ([_vp, _vp, _i, _vp, _vp, _d, _i, _i, ctypes.POINTER(SolveInfo), _vp], _i),
    "hqmc_estimate_multi": ([_vp, _vp, ctypes.c_uint64, ctypes.c_uint64, _i, _d, _i, _i, _vp, _vp,
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolveInfo), _vp], _i),
    "hqmc_force": ([_vp, _vp, _vp, _vp, _vp, _vp], _i),
    "hqmc_action_terms": ([_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double), _vp], _i),
    "hqmc_draw": ([_vp, _u64, _u64, _vp, _vp, ctypes.POINTER(ctypes.c_double), _vp], _i),
    "hqmc_leapfrog": ([_vp, _vp, _vp, _vp, _vp, _i, _d, _d, _i, _i, ctypes.POINTER(TrajInfo), _vp], _i),
    "hqmc_trajectory": ([_vp, _vp, _u64, _u64, _vp, _vp, ctypes.POINTER(ctypes.c_double), _i, _d, _d, _i, _i,
                         ctypes.POINTER(TrajInfo), _vp], _i),
    "hqmc_set_timing": ([_vp, _i], _i),
    "hqmc_get_timing": ([_vp, _i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)], _i),
    "hqmc_get_timing_samples": ([_vp, _i, ctypes.POINTER(ctypes.c_float), _i, ctypes.POINTER(_i)], _i),
    "hqmc_probe_fp64_rate": ([_vp, ctypes.POINTER(ctypes.c_double)], _i),
    "hqmc_apply_MdagM_static": ([ctypes.POINTER(Params), _vp, _vp, _vp, _vp], _i),
    "hqmc_make_batch": ([ctypes.POINTER(Params), _i, ctypes.POINTER(_vp)], _i),
    "hqmc_free_batch": ([_vp], _i),
    "hqmc_batch_last_error": ([_vp], ctypes.c_char_p),
    "hqmc_batch_launch_count": ([_vp], ctypes.c_longlong),
    "hqmc_batch_set_solver": ([_vp, _i], _i),
    "hqmc_batch_launch_shape": ([_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                                 ctypes.POINTER(ctypes.c_float)], _i),
    "hqmc_batch_cg_solve": ([_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _d, _i,
                             ctypes.POINTER(SolveInfo), _vp], _i),
    "hqmc_batch_trajectory": ([_vp, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_uint64), _u64, _i,
                               ctypes.POINTER(ctypes.c_double), _d, _i, ctypes.POINTER(TrajInfo), _vp], _i),
    "hqmc_net_create": ([_u64, ctypes.POINTER(_vp)], _i),
    "hqmc_net_free": ([_vp], _i),
    "hqmc_net_num_weights": ([_vp], _i),
    "hqmc_net_get_weights": ([_vp, ctypes.POINTER(ctypes.c_float), _i], _i),
    "hqmc_net_set_weights": ([_vp, ctypes.POINTER(ctypes.c_float), _i], _i),
    "hqmc_net_apply": ([_vp, _vp, _vp, _vp, _vp, _vp], _i),
    "hqmc_net_train_step": ([_vp, _vp, _vp, _vp, _vp, _d, ctypes.POINTER(ctypes.c_double), _vp], _i),
    "hqmc_set_preconditioner": ([_vp, _vp], _i),
    "hqmc_set_net_interval": ([_vp, _i], _i),
    "hqmc_set_net_tensor_cores": ([_vp, _i], _i),
    "hqmc_set_guess_history": ([_vp, _i], _i),
    "hqmc_checkpoint_write": ([ctypes.c_char_p, ctypes.POINTER(Checkpoint), _vp, _vp], _i),
    "hqmc_checkpoint_read": ([ctypes.c_char_p, ctypes.POINTER(Checkpoint), _vp, _vp], _i),
}
for _name, (_args, _res) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class HQMCError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        msg = _lib.hqmc_strerror(status).decode()
        super().__init__(f"{msg} ({status})" + (f": {detail}" if detail else ""))


def strerror(status: int) -> str:
    return _lib.hqmc_strerror(status).decode()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


class Config:
    """Owns an hqmc_config: lattice, model parameters, launch shapes and workspace."""

    def __init__(self, L: int, Ntau: int, dtau: float = 0.1, t: float = 1.0, J: float = 1.0,
                 K: float = 0.0, noncompact: bool = False, reliable_interval: int = 50, autotune: bool = False,
                 variant: int = 0):
        self.params = Params(L, Ntau, dtau, t, J, K, ACTION_NONCOMPACT if noncompact else ACTION_COMPACT,
                             reliable_interval, int(autotune), variant)
        h = _vp()
        rc = _lib.hqmc_make_config(ctypes.byref(self.params), ctypes.byref(h))
        if rc != OK:
            raise HQMCError(rc, f"L={L} Ntau={Ntau}")
        self._h = h
        self.L, self.Ntau = L, Ntau
        self.n_sites = int(_lib.hqmc_num_sites(h))

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("config already freed")
        return self._h

    def launch_shape(self, precision: int = FP64) -> dict:
        """Fused M^dagger M launch shape chosen for a precision (see hqmc_get_launch_shape)."""
        v, c, t, us = _i(), _i(), _i(), ctypes.c_float()
        self.check(_lib.hqmc_get_launch_shape(self.handle, precision, ctypes.byref(v), ctypes.byref(c),
                                              ctypes.byref(t), ctypes.byref(us)))
        return {"variant": v.value, "cluster": c.value, "threads": t.value, "tuned_us": us.value}

    def launch_count(self) -> int:
        """Kernels this config has enqueued so far."""
        return int(_lib.hqmc_launch_count(self.handle))

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.hqmc_free_config(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def check(self, rc: int, allow=(OK,)):
        if rc not in allow:
            raise HQMCError(rc, (_lib.hqmc_last_error(self._h) or b"").decode())
        return rc

    # -- argument checks ---------------------------------------------------
    def _bonds(self, a, name):
        if a is None:
            return None
        if not (a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()
                and tuple(a.shape) == (self.Ntau, self.L, self.L, 2)):
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of shape "
                             f"({self.Ntau}, {self.L}, {self.L}, 2)")
        return a

    def _vec(self, a, name, dtypes=(torch.complex128,)):
        if a is None:
            return None
        if not (a.is_cuda and a.dtype in dtypes and a.is_contiguous()
                and tuple(a.shape) == (self.Ntau, self.L, self.L)):
            raise ValueError(f"{name} must be a contiguous CUDA tensor of dtype {dtypes} and shape "
                             f"({self.Ntau}, {self.L}, {self.L})")
        return a

    def empty_vec(self, dtype=torch.complex128):
        return torch.empty((self.Ntau, self.L, self.L), dtype=dtype, device="cuda")

    def empty_bonds(self):
        return torch.empty((self.Ntau, self.L, self.L, 2), dtype=torch.float64, device="cuda")


def make_config(L: int, Ntau: int, **kw) -> Config:
    return Config(L, Ntau, **kw)


def _prec(x) -> int:
    return FP32 if x.dtype == torch.complex64 else FP64


def apply_M(cfg: Config, theta, x, y=None, dagger: bool = False):
    """y = M x (or M^dagger x); complex64 x selects the FP32 kernel."""
    cfg._bonds(theta, "theta")
    cfg._vec(x, "x", (torch.complex128, torch.complex64))
    y = torch.empty_like(x) if y is None else cfg._vec(y, "y", (x.dtype,))
    cfg.check(_lib.hqmc_apply_M(cfg.handle, _ptr(theta), _ptr(x), _ptr(y), int(dagger), _prec(x), _stream()))
    return y


def apply_MdagM(cfg: Config, theta, x, y=None):
    """y = (M^dagger M) x with the fused kernel; complex64 x selects FP32."""
    cfg._bonds(theta, "theta")
    cfg._vec(x, "x", (torch.complex128, torch.complex64))
    y = torch.empty_like(x) if y is None else cfg._vec(y, "y", (x.dtype,))
    cfg.check(_lib.hqmc_apply_MdagM(cfg.handle, _ptr(theta), _ptr(x), _ptr(y), _prec(x), _stream()))
    return y


def apply_precond(cfg: Config, r, z=None):
    """z = Otilde^{-1} r, the tau-line preconditioner; complex64 r selects FP32."""
    cfg._vec(r, "r", (torch.complex128, torch.complex64))
    z = torch.empty_like(r) if z is None else cfg._vec(z, "z", (r.dtype,))
    cfg.check(_lib.hqmc_apply_precond(cfg.handle, _ptr(r), _ptr(z), _prec(r), _stream()))
    return z


def get_precond(cfg: Config) -> dict:
    """Coefficients of the tau-line preconditioner: a, b (pi-flux O), rho, W."""
    a, b, rho, W = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), _i()
    cfg.check(_lib.hqmc_get_precond(cfg.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(rho),
                                    ctypes.byref(W)))
    return {"a": a.value, "b": b.value, "rho": rho.value, "W": W.value}


def get_precond_shape(cfg: Config, precision: int = FP32) -> dict:
    """Preconditioner launch shape: slices per tile of the separate kernel, and
    whether preconditioned CG fuses the update with the preconditioner."""
    tc, fused = _i(), _i()
    cfg.check(_lib.hqmc_get_precond_shape(cfg.handle, precision, ctypes.byref(tc), ctypes.byref(fused)))
    return {"tile_slices": tc.value, "fused": bool(fused.value)}


def set_precond_fused(cfg: Config, fused: bool, precision: int = FP32):
    """Force the fused (True) or separate (False) preconditioned CG update for one precision."""
    cfg.check(_lib.hqmc_set_precond_fused(cfg.handle, precision, int(fused)))


def _solver(s) -> int:
    if isinstance(s, str):
        return SOLVERS[s]
    return int(s)


def cg_solve(cfg: Config, theta, phi, x=None, tol: float = 1e-8, maxit: int = 100000, solver="cg64",
             raise_on_fail: bool = True):
    """Solve (M^dagger M) x = phi.  Returns (x, info dict).  x (if given) is the initial guess."""
    cfg._bonds(theta, "theta")
    cfg._vec(phi, "phi")
    x = torch.zeros_like(phi) if x is None else cfg._vec(x, "x")
    info = SolveInfo()
    rc = _lib.hqmc_cg_solve(cfg.handle, _ptr(theta), _ptr(phi), _ptr(x), tol, maxit, _solver(solver),
                            ctypes.byref(info), _stream())
    if raise_on_fail:
        cfg.check(rc)
    return x, info.as_dict()


def set_multi_rhs(cfg: Config, nmax: int):
    """Workspace for up to nmax systems solved together on one field (hqmc_set_multi_rhs;
    0 frees it)."""
    cfg.check(_lib.hqmc_set_multi_rhs(cfg.handle, nmax))


def set_multi_ranges(cfg: Config, ranges: int):
    """Slice ranges per system of the multi-system walk launch (0: the default model)."""
    cfg.check(_lib.hqmc_set_multi_ranges(cfg.handle, ranges))


def multi_launch_shape(cfg: Config, nrhs: int) -> dict:
    """Slice ranges per system, block size and strip height of a multi-system solve."""
    r, t, b = _i(), _i(), _i()
    cfg.check(_lib.hqmc_multi_launch_shape(cfg.handle, nrhs, ctypes.byref(r), ctypes.byref(t), ctypes.byref(b)))
    return {"ranges": r.value, "threads": t.value, "nby": b.value}


def cg_solve_multi(cfg: Config, theta, phi, x=None, tol: float = 1e-8, maxit: int = 100000, solver="pmixed",
                   raise_on_fail: bool = True):
    """Solve (M^dagger M) x_k = phi_k for the nrhs systems of phi (shape (nrhs, Ntau, L, L))
    together (hqmc_cg_solve_multi; needs set_multi_rhs(cfg, >= nrhs)).  Returns (x, infos)."""
    cfg._bonds(theta, "theta")
    if phi.dim() != 4 or tuple(phi.shape[1:]) != (cfg.Ntau, cfg.L, cfg.L) or phi.dtype != torch.complex128 \
            or not phi.is_contiguous():
        raise ValueError("phi must be a contiguous complex128 tensor of shape (nrhs, Ntau, L, L)")
    x = torch.zeros_like(phi) if x is None else x
    if x.shape != phi.shape or x.dtype != phi.dtype or not x.is_contiguous():
        raise ValueError("x must match phi")
    nrhs = phi.shape[0]
    infos = (SolveInfo * nrhs)()
    rc = _lib.hqmc_cg_solve_multi(cfg.handle, _ptr(theta), nrhs, _ptr(phi), _ptr(x), tol, maxit, _solver(solver),
                                  infos, _stream())
    if raise_on_fail:
        cfg.check(rc)
    return x, [i.as_dict() for i in infos]


def estimate(cfg: Config, theta, nrv: int, seed: int = 0, counter: int = 0, tol: float = 1e-8,
             maxit: int = 100000, solver="cg64", want_vectors: bool = False, raise_on_fail: bool = True,
             projected: bool = False, Gxi=None, together: bool = False):
    """Stochastic estimation with nrv CN(0, 1) vectors (hqmc_estimate; with
    projected=True hqmc_estimate_projected, which needs the solutions: Gxi is then
    allocated here unless given; with together=True hqmc_estimate_multi, the systems
    solved together, which needs set_multi_rhs).  Returns (g, infos, Gxi, xi): g the
    complex estimate of the mean diagonal of M^{-1}, the per-vector solve infos, and
    (if want_vectors) M^{-1} xi_k and xi_k as tensors of shape (nrv, Ntau, L, L)."""
    if projected and together:
        raise ValueError("projected and together are different estimates")
    cfg._bonds(theta, "theta")
    xi = None
    if Gxi is None and (want_vectors or projected):
        Gxi = torch.empty((nrv, cfg.Ntau, cfg.L, cfg.L), dtype=torch.complex128, device=theta.device)
    if want_vectors:
        xi = torch.empty_like(Gxi)
    g = (ctypes.c_double * 2)()
    infos = (SolveInfo * nrv)()
    fn = _lib.hqmc_estimate_projected if projected else _lib.hqmc_estimate_multi if together else _lib.hqmc_estimate
    rc = fn(cfg.handle, _ptr(theta), seed, counter, nrv, tol, maxit, _solver(solver), _ptr(Gxi), _ptr(xi), g, infos,
            _stream())
    if raise_on_fail:
        cfg.check(rc, allow=(OK, ENOTCONV))
    return complex(g[0], g[1]), [i.as_dict() for i in infos], Gxi, xi


def force(cfg: Config, theta, X, F=None, dSf=None):
    """Total force F = -dS_B/dtheta - dS_f/dtheta given X = (M^dagger M)^{-1} phi."""
    cfg._bonds(theta, "theta")
    cfg._vec(X, "X")
    F = cfg.empty_bonds() if F is None else cfg._bonds(F, "F")
    cfg._bonds(dSf, "dSf")
    cfg.check(_lib.hqmc_force(cfg.handle, _ptr(theta), _ptr(X), _ptr(F), _ptr(dSf), _stream()))
    return F


def action_terms(cfg: Config, theta, p=None, phi=None, X=None):
    """(S_B, sum p^2, Re phi^dagger X) of Eq. (H_hmc)."""
    cfg._bonds(theta, "theta")
    cfg._bonds(p, "p")
    cfg._vec(phi, "phi")
    cfg._vec(X, "X")
    out = (ctypes.c_double * 3)()
    cfg.check(_lib.hqmc_action_terms(cfg.handle, _ptr(theta), _ptr(p), _ptr(phi), _ptr(X), out, _stream()))
    return out[0], out[1], out[2]


def draw(cfg: Config, seed: int, traj_counter: int, p=None, R=None, want_p: bool = True, want_R: bool = True):
    """Philox draws of HQMC step (i): p ~ N(0, 1/2) per bond, R ~ CN(0, 1) per site, and u."""
    if want_p and p is None:
        p = cfg.empty_bonds()
    if want_R and R is None:
        R = cfg.empty_vec()
    cfg._bonds(p, "p")
    cfg._vec(R, "R")
    u = ctypes.c_double()
    cfg.check(_lib.hqmc_draw(cfg.handle, seed, traj_counter, _ptr(p), _ptr(R), ctypes.byref(u), _stream()))
    return p, R, u.value


def leapfrog(cfg: Config, theta, p, phi, X, nsteps: int, dt: float, tol: float = 1e-8, maxit: int = 100000,
             solver="cg64"):
    """nsteps leapfrog steps on (theta, p) in place; X is the CG guess in and the solution out."""
    cfg._bonds(theta, "theta")
    cfg._bonds(p, "p")
    cfg._vec(phi, "phi")
    cfg._vec(X, "X")
    info = TrajInfo()
    cfg.check(_lib.hqmc_leapfrog(cfg.handle, _ptr(theta), _ptr(p), _ptr(phi), _ptr(X), nsteps, dt, tol, maxit,
                                 _solver(solver), ctypes.byref(info), _stream()), allow=(OK, ENOTCONV))
    return info.as_dict()


def trajectory(cfg: Config, theta, seed: int = 0, traj_counter: int = 0, p_in=None, R_in=None, u_in=None,
               nsteps: int = 10, dt: float = 0.05, tol: float = 1e-8, maxit: int = 100000, solver="cg64"):
    """One HQMC update of theta (in place).  Returns the trajectory info dict."""
    cfg._bonds(theta, "theta")
    cfg._bonds(p_in, "p_in")
    cfg._vec(R_in, "R_in")
    info = TrajInfo()
    u = None if u_in is None else ctypes.byref(ctypes.c_double(u_in))
    cfg.check(_lib.hqmc_trajectory(cfg.handle, _ptr(theta), seed, traj_counter, _ptr(p_in), _ptr(R_in), u,
                                   nsteps, dt, tol, maxit, _solver(solver), ctypes.byref(info), _stream()),
              allow=(OK, ENOTCONV))
    return info.as_dict()


def set_timing(cfg: Config, enable: bool):
    cfg.check(_lib.hqmc_set_timing(cfg.handle, int(enable)))


def get_timing(cfg: Config, timer: int):
    """(launches, total milliseconds) of one kernel class since set_timing."""
    n, ms = ctypes.c_longlong(), ctypes.c_double()
    cfg.check(_lib.hqmc_get_timing(cfg.handle, timer, ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def get_timing_samples(cfg: Config, timer: int) -> list:
    """Per-launch durations (microseconds) of one kernel class since set_timing, in launch order."""
    n = _i()
    cfg.check(_lib.hqmc_get_timing_samples(cfg.handle, timer, None, 0, ctypes.byref(n)))
    buf = (ctypes.c_float * max(n.value, 1))()
    cfg.check(_lib.hqmc_get_timing_samples(cfg.handle, timer, buf, n.value, ctypes.byref(n)))
    return list(buf[:n.value])


def probe_fp64_rate(cfg: Config) -> float:
    """Measured FP64 FMA throughput of the current device in TFLOP/s."""
    out = ctypes.c_double()
    cfg.check(_lib.hqmc_probe_fp64_rate(cfg.handle, ctypes.byref(out)))
    return out.value


STATIC_MAX_SITES = 262144


def apply_MdagM_static(L: int, Ntau: int, theta, x, y=None, dtau: float = 0.1, t: float = 1.0):
    """y = (M^dagger M) x in FP64 through hqmc_apply_MdagM_static: no config and no
    device allocation inside the library, for callers that cannot allocate
    (scratch is a fixed device array of STATIC_MAX_SITES sites; calls on one
    device must not overlap on the GPU).  Returns y; raises HQMCError on failure."""
    shape = (Ntau, L, L)
    if not (theta.is_cuda and theta.dtype == torch.float64 and theta.is_contiguous()
            and tuple(theta.shape) == shape + (2,)):
        raise ValueError("theta must be a contiguous CUDA float64 tensor of shape (Ntau, L, L, 2)")
    if not (x.is_cuda and x.dtype == torch.complex128 and x.is_contiguous() and tuple(x.shape) == shape):
        raise ValueError("x must be a contiguous CUDA complex128 tensor of shape (Ntau, L, L)")
    y = torch.empty_like(x) if y is None else y
    p = Params(L, Ntau, dtau, t, 1.0, 0.0, ACTION_COMPACT, 0, 0, 0)
    rc = _lib.hqmc_apply_MdagM_static(ctypes.byref(p), _ptr(theta), _ptr(x), _ptr(y), _stream())
    if rc != OK:
        raise HQMCError(rc, f"static apply at L={L} Ntau={Ntau}")
    return y


class Batch:
    """Independent chains of possibly different lattices driven together (hqmc_make_batch)."""

    def __init__(self, lattices, dtau: float = 0.1, t: float = 1.0, J: float = 1.0, K: float = 0.0,
                 noncompact: bool = False, autotune: bool = False):
        self.lattices = [(int(L), int(N)) for L, N in lattices]
        n = len(self.lattices)
        arr = (Params * n)(*[Params(L, N, dtau, t, J, K, ACTION_NONCOMPACT if noncompact else ACTION_COMPACT,
                                    0, 1 if autotune else 0, 1) for L, N in self.lattices])
        h = _vp()
        rc = _lib.hqmc_make_batch(arr, n, ctypes.byref(h))
        if rc != OK:
            raise HQMCError(rc, "batch creation")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.hqmc_free_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def launch_count(self) -> int:
        return int(_lib.hqmc_batch_launch_count(self._h))

    def launch_shape(self) -> dict:
        """Tile shape of the batched fused launch (hqmc_batch_launch_shape)."""
        c, o, t, us = _i(), _i(), _i(), ctypes.c_float()
        self._check(_lib.hqmc_batch_launch_shape(self._h, ctypes.byref(c), ctypes.byref(o), ctypes.byref(t),
                                                 ctypes.byref(us)))
        return {"cluster": c.value, "order": o.value, "threads": t.value, "tuned_us": us.value}

    def set_solver(self, solver):
        """"cg64" (default) or "pcg64" for every chain (hqmc_batch_set_solver)."""
        self._check(_lib.hqmc_batch_set_solver(self._h, _solver(solver)))

    def _check(self, rc, allow=(OK,)):
        if rc not in allow:
            raise HQMCError(rc, (_lib.hqmc_batch_last_error(self._h) or b"").decode())

    def _ptrs(self, tensors):
        return (_vp * len(tensors))(*[t.data_ptr() for t in tensors])

    def cg_solve(self, thetas, phis, xs=None, tol: float = 1e-8, maxit: int = 100000, raise_on_fail: bool = True):
        n = len(self.lattices)
        xs = [torch.zeros_like(p) for p in phis] if xs is None else xs
        infos = (SolveInfo * n)()
        rc = _lib.hqmc_batch_cg_solve(self._h, self._ptrs(thetas), self._ptrs(phis), self._ptrs(xs), tol, maxit,
                                      infos, _stream())
        if raise_on_fail:
            self._check(rc)
        return xs, [i.as_dict() for i in infos]

    def trajectory(self, thetas, seeds, traj_counter: int, nsteps: int, dts, tol: float = 1e-8,
                   maxit: int = 100000):
        n = len(self.lattices)
        infos = (TrajInfo * n)()
        rc = _lib.hqmc_batch_trajectory(self._h, self._ptrs(thetas), (ctypes.c_uint64 * n)(*seeds), traj_counter,
                                        nsteps, (ctypes.c_double * n)(*dts), tol, maxit, infos, _stream())
        self._check(rc, allow=(OK, ENOTCONV))
        return [i.as_dict() for i in infos]


class Net:
    """Learned preconditioner K(theta) (hqmc_net_*): 4 gauge-covariant linear stencil layers,
    1 -> 16 -> 16 -> 16 -> 1 complex channels, BF16 weights, FP32 arithmetic."""

    def __init__(self, seed: int = 0):
        h = _vp()
        rc = _lib.hqmc_net_create(seed, ctypes.byref(h))
        if rc != OK:
            raise HQMCError(rc, "net creation")
        self._h = h
        self.n_weights = int(_lib.hqmc_net_num_weights(h))

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.hqmc_net_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_weights(self):
        import numpy as np
        w = np.empty(self.n_weights, dtype=np.float32)
        rc = _lib.hqmc_net_get_weights(self._h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self.n_weights)
        if rc != OK:
            raise HQMCError(rc, "get weights")
        return w

    def set_weights(self, w):
        import numpy as np
        w = np.ascontiguousarray(w, dtype=np.float32)
        rc = _lib.hqmc_net_set_weights(self._h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), w.size)
        if rc != OK:
            raise HQMCError(rc, "set weights")

    def apply(self, cfg: Config, theta, r, z=None):
        cfg._bonds(theta, "theta")
        cfg._vec(r, "r")
        z = torch.empty_like(r) if z is None else cfg._vec(z, "z")
        cfg.check(_lib.hqmc_net_apply(cfg.handle, self._h, _ptr(theta), _ptr(r), _ptr(z), _stream()))
        return z

    def train_step(self, cfg: Config, theta, phi, x, lr: float = 1e-3, want_loss: bool = True):
        cfg._bonds(theta, "theta")
        cfg._vec(phi, "phi")
        cfg._vec(x, "x")
        loss = ctypes.c_double()
        cfg.check(_lib.hqmc_net_train_step(cfg.handle, self._h, _ptr(theta), _ptr(phi), _ptr(x), lr,
                                           ctypes.byref(loss) if want_loss else None, _stream()))
        return loss.value if want_loss else None


def set_preconditioner(cfg: Config, net):
    """Attach (or with None detach) the net of the learned solvers; the first attach
    allocates the config's net workspace."""
    cfg.check(_lib.hqmc_set_preconditioner(cfg.handle, None if net is None else net.handle))


def set_guess_history(cfg: Config, k: int):
    """Chronological initial guess of leapfrog solves from the last k solutions
    (hqmc_set_guess_history; 0 = the previous solution)."""
    cfg.check(_lib.hqmc_set_guess_history(cfg.handle, int(k)))


def set_net_interval(cfg: Config, k: int):
    """Flexible CG ("flearned"): the net preconditions every k-th iteration, the
    tau-line preconditioner the others."""
    cfg.check(_lib.hqmc_set_net_interval(cfg.handle, int(k)))


def set_net_tensor_cores(cfg: Config, on: bool):
    """Inference 16 -> 16 layers on tensor cores (BF16 operands, FP32 accumulation;
    the default) or in FP32 on CUDA cores."""
    cfg.check(_lib.hqmc_set_net_tensor_cores(cfg.handle, 1 if on else 0))


def save_checkpoint(path: str, theta, seed: int, traj_counter: int, dt: float, nsteps: int, solver="cg64",
                    trajectories: int = 0, accepted: int = 0, dtau: float = 0.1, t: float = 1.0, J: float = 1.0,
                    K: float = 0.0, noncompact: bool = False, net=None):
    """Write a chain checkpoint (hqmc_checkpoint_write): theta (CPU or CUDA float64
    tensor of shape (Ntau, L, L, 2)) is copied to host memory first."""
    import numpy as np
    th = np.ascontiguousarray(theta.detach().cpu().numpy(), dtype=np.float64)
    Ntau, L = th.shape[0], th.shape[1]
    w = net.get_weights() if net is not None else None
    c = Checkpoint(L, Ntau, dtau, t, J, K, ACTION_NONCOMPACT if noncompact else ACTION_COMPACT,
                   0 if w is None else w.size, seed, traj_counter, dt, nsteps, _solver(solver), trajectories,
                   accepted, 1, 0)
    rc = _lib.hqmc_checkpoint_write(path.encode(), ctypes.byref(c), th.ctypes.data,
                                    None if w is None else w.ctypes.data)
    if rc != OK:
        raise HQMCError(rc, path)


def load_checkpoint(path: str):
    """Read a chain checkpoint (hqmc_checkpoint_read).  Returns (header dict, theta as a
    CPU float64 tensor, net weights as a float32 numpy array or None)."""
    import numpy as np
    c = Checkpoint()
    rc = _lib.hqmc_checkpoint_read(path.encode(), ctypes.byref(c), None, None)
    if rc != OK:
        raise HQMCError(rc, path)
    th = np.empty((c.Ntau, c.L, c.L, 2), dtype=np.float64)
    w = np.empty(c.n_weights, dtype=np.float32) if c.n_weights else None
    rc = _lib.hqmc_checkpoint_read(path.encode(), ctypes.byref(c), th.ctypes.data, None if w is None else w.ctypes.data)
    if rc != OK:
        raise HQMCError(rc, path)
    return c.as_dict(), torch.from_numpy(th), w


def log_trajectory(fp, info: dict, **extra):
    """Append one JSON line for a trajectory (its info dict plus any extra fields,
    e.g. the step time) to an open text file."""
    import json
    fp.write(json.dumps(dict(info, **extra)) + "\n")
    fp.flush()
