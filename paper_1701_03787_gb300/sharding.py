"""Mode sharding across ranks (host logic only).

The solves of different Fourier modes are independent (Sec. 4: one serial solve per
mode; the paper's MPI exchange sits in the transforms, not in the solves).  A field
of n_modes columns is split into contiguous ranges, one per rank; each rank solves
its range with ``shen_solve_modes`` on its own GPU.  There is no collective on the
data path.
"""


def shard_range(n_modes, rank, world):
    """(mode_begin, mode_count) of `rank`'s contiguous share of n_modes modes; the
    first n_modes % world ranks take one mode more."""
    if world < 1 or not 0 <= rank < world or n_modes < 0:
        raise ValueError("need 0 <= rank < world and n_modes >= 0")
    base, extra = divmod(n_modes, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def solve_shard(plan, problem, f, u=None, rank=0, world=1, precision="fp64", stream=None):
    """Solve this rank's modes of the plan.  f (and u): DEVICE tensors holding only
    this rank's columns, shape (count, N)."""
    begin, count = shard_range(plan.n_modes, rank, world)
    if f.shape[0] != count:
        raise ValueError(f"rank {rank} holds {count} modes, f has {f.shape[0]}")
    return plan.solve_modes(problem, begin, f, u, precision=precision, stream=stream)
