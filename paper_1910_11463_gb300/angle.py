"""Angular decomposition of source iteration (Sec. 5, parallel in angle).

Every process holds the whole mesh and a contiguous block of the quadrature's
directions with their hierarchies; once per source iteration the scalar flux,
a quadrature sum over directions (Eq. angular_quad), is summed over the
processes.  libpair does that through the reduction function of si_params
(pair_reduce_fn): between its partial quadrature sum and its convergence test it
hands the partial flux and a status value to the function, which sums them over
the processes (here torch.distributed.all_reduce), so every process continues
with the same flux and takes the same stopping decision."""
from __future__ import annotations

import numpy as np


def direction_block(M: int, world: int, rank: int) -> tuple[int, int]:
    """Directions [m0, m1) of `rank` when M directions are split over `world`
    processes in contiguous blocks whose sizes differ by at most one (the first
    M % world processes take one more)."""
    if not (0 <= rank < world) or M < world:
        raise ValueError(f"cannot split {M} directions over {world} processes (rank {rank})")
    base, extra = divmod(M, world)
    m0 = rank * base + min(rank, extra)
    return m0, m0 + base + (1 if rank < extra else 0)


def allreduce_sum(group=None):
    """Reduction for si_solve's phi_reduce: in-place sum over the process group."""
    import torch.distributed as dist

    def fn(v):
        dist.all_reduce(v, op=dist.ReduceOp.SUM, group=group)
    return fn


def si_solve_angle(geom, omega, w, sigma_t, sigma_s, q, rank: int, world: int, reduce=None, **kw):
    """si_solve on this process's block of directions, the scalar flux summed over
    the processes every iteration (default: torch.distributed all-reduce on the
    default group).  Returns (phi of the whole quadrature, psi of this block or
    None, info of this process, (m0, m1))."""
    from . import pair
    om = np.ascontiguousarray(omega, dtype=np.float64)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    m0, m1 = direction_block(len(ww), world, rank)
    phi, psi, info = pair.si_solve(geom, om[m0:m1], ww[m0:m1], sigma_t, sigma_s, q,
                                   phi_reduce=reduce if reduce is not None else allreduce_sum(), **kw)
    return phi, psi, info, (m0, m1)
