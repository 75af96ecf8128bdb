"""Imaginary-time slab decomposition of the HQMC operator over several ranks.

The fermion matrix couples slice tau only to tau - 1 (Methods, Eq. (M_alpha)),
so M^dagger M couples tau to tau - 1, tau and tau + 1, and the pseudofermion
force on slice tau needs X_tau and X_{tau+1} (Supplement SI).  A rank that holds
the contiguous slices [tau0, tau1) of theta and of every vector therefore needs
one halo slice of the vector on each side per operator application, and theta
on one slice on each side once per field; the CG inner products are sums over
the ranks.

Antiperiodic boundary: the halo slices are received already multiplied by the
boundary sign where they cross the global wrap (the slice left of tau = 0 is
-x_{Ntau-1}, the slice right of tau = Ntau - 1 is -x_0).  Every row of the
extended slab [tau0 - 1, tau1] other than its two ends is then an ordinary
interior row of M^dagger M (and of the force) on a lattice of n_local + 2
slices: (M x)_0 = x_0 + B x_{Ntau-1} = x_0 - B (-x_{Ntau-1}).  So the per-rank
operator is the library's own apply and force on a config of n_local + 2 slices
(`LibrarySlabOperator`), and rows 1..n_local of its output are the rank's rows.
theta is periodic in tau and its halos carry no sign.

Collectives: `halo` exchanges one slice with each neighbour (point-to-point,
isend/irecv), `allreduce_sum` sums the CG scalars; both go through
torch.distributed (NCCL between GPUs, gloo on CPU).  With one rank the halos
come from the rank's own ends.  The vector algebra of the distributed CG is done
on the rank's tensors.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch


@dataclass(frozen=True)
class SlabLayout:
    """Contiguous, balanced slabs: rank r holds slices [tau0, tau1)."""

    Ntau: int
    world: int
    rank: int

    @property
    def tau0(self) -> int:
        return self.rank * self.Ntau // self.world

    @property
    def tau1(self) -> int:
        return (self.rank + 1) * self.Ntau // self.world

    @property
    def n_local(self) -> int:
        return self.tau1 - self.tau0

    @property
    def left(self) -> int:
        return (self.rank - 1) % self.world

    @property
    def right(self) -> int:
        return (self.rank + 1) % self.world


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def allreduce_sum(v: torch.Tensor) -> torch.Tensor:
    """Sum of a small tensor over the ranks (in place; returned)."""
    dist = _dist()
    if dist is not None and dist.get_world_size() > 1:
        dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return v


def halo(local: torch.Tensor, lay: SlabLayout, antiperiodic: bool) -> torch.Tensor:
    """The rank's slices with one neighbour slice on each side (shape (n_local + 2, ...)).
    antiperiodic: the halo slices that cross the global wrap are negated (vectors);
    theta is periodic (antiperiodic=False)."""
    ext = torch.empty((local.shape[0] + 2,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    ext[1:-1] = local
    dist = _dist()
    if lay.world == 1 or dist is None:
        ext[0] = local[-1]
        ext[-1] = local[0]
    else:
        first = local[0].contiguous()
        last = local[-1].contiguous()
        recv_l = torch.empty_like(first)
        recv_r = torch.empty_like(first)
        # tag 0: a rank's last slice travels right; tag 1: its first slice travels left
        reqs = [dist.isend(last, lay.right, tag=0), dist.irecv(recv_l, lay.left, tag=0),
                dist.isend(first, lay.left, tag=1), dist.irecv(recv_r, lay.right, tag=1)]
        for r in reqs:
            r.wait()
        ext[0] = recv_l
        ext[-1] = recv_r
    if antiperiodic:
        if lay.tau0 == 0:
            ext[0] = -ext[0]
        if lay.tau1 == lay.Ntau:
            ext[-1] = -ext[-1]
    return ext


class LibrarySlabOperator:
    """The rank's operator: the library's fused M^dagger M and force on a config of
    n_local + 2 slices (rows 1..n_local are the rank's rows)."""

    def __init__(self, L: int, n_local: int, **params):
        from . import hqmc
        self.hqmc = hqmc
        self.cfg = hqmc.Config(L, n_local + 2, **params)

    def apply_MdagM_ext(self, theta_ext, x_ext):
        return self.hqmc.apply_MdagM(self.cfg, theta_ext, x_ext)

    def force_ext(self, theta_ext, X_ext):
        """Total force -dS_B/dtheta - dS_f/dtheta on the extended slab."""
        return self.hqmc.force(self.cfg, theta_ext, X_ext)

    def close(self):
        self.cfg.close()


def apply_MdagM(op, theta_ext, x_local, lay: SlabLayout):
    """Rows [tau0, tau1) of (M^dagger M) x."""
    return op.apply_MdagM_ext(theta_ext, halo(x_local, lay, True))[1:-1]


def _rdot(a, b) -> torch.Tensor:
    return torch.sum(a.real * b.real + a.imag * b.imag).reshape(1).to(torch.float64)


def cg(op, theta_ext, phi_local, x_local, lay: SlabLayout, tol: float = 1e-8, maxit: int = 100000):
    """CG on (M^dagger M) X = phi over the slabs (Eq. (pCG) with the identity
    preconditioner): one halo exchange per operator application, the inner products
    summed over the ranks.  Stops on the true residual ||phi - O X|| <= tol ||phi||,
    restarting from it if the recursion drifted.  x_local is updated in place.
    Returns (iterations, true relative residual)."""
    bb = allreduce_sum(_rdot(phi_local, phi_local)).item()
    if bb == 0.0:
        x_local.zero_()
        return 0, 0.0
    k = 0
    while True:
        r = phi_local - apply_MdagM(op, theta_ext, x_local, lay)
        rr = allreduce_sum(_rdot(r, r)).item()
        if rr <= tol * tol * bb or k >= maxit:
            return k, (rr / bb) ** 0.5
        p = r.clone()
        while k < maxit:
            q = apply_MdagM(op, theta_ext, p, lay)
            pq = allreduce_sum(_rdot(p, q)).item()
            alpha = rr / pq
            x_local += alpha * p
            r -= alpha * q
            k += 1
            rr_new = allreduce_sum(_rdot(r, r)).item()
            if rr_new <= tol * tol * bb:
                break
            p = r + (rr_new / rr) * p
            rr = rr_new


def force(op, theta_ext, X_local, lay: SlabLayout):
    """Rows [tau0, tau1) of the total force F = -dS_B/dtheta - dS_f/dtheta given
    X = (M^dagger M)^{-1} phi: the fermion part needs X on the next slice (halo),
    the bosonic part theta on both neighbouring slices (theta_ext)."""
    return op.force_ext(theta_ext, halo(X_local, lay, True))[1:-1]
