"""Non-LTE iteration with its wavelengths split between processes (one GPU each).

Within an iteration the wavelengths are independent (Sec. 3.6): rank r runs the formal
solution of a contiguous range of the atom's grid wavelengths and reduces it to the two
radiation integrals per line and cell that the rates of Sec. 3.3 need (rc_line_integrals).
One all-reduce (sum) of those n_lines x 2 FP64 values per cell gives every rank the
integrals over all wavelengths; each rank then solves the statistical equilibrium of every
cell (rc_stat_eq_integrals) and, holding the same sums, ends the iteration with the same
populations and the same maximum change.  The all-reduce is the method's one exchange step.

``nlte_solve_sharded`` strings the steps together through an ``ops`` object:
``GpuOps`` calls librcx.so; any object with the same four methods can stand in for it.
"""
from __future__ import annotations


def lambda_range(rank: int, world: int, n_lambda: int) -> tuple[int, int]:
    """(begin, count) of rank's contiguous share of n_lambda wavelengths; the first
    n_lambda % world ranks take one more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    base, extra = divmod(n_lambda, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


class GpuOps:
    """The steps of one iteration through the library (device tensors, the current stream)."""

    def __init__(self, plan, atom, T, ne, n_atom):
        self.plan, self.atom = plan, atom
        self.T, self.ne, self.n_atom = T.reshape(-1), ne, n_atom

    def emis_opac(self, pops):
        return self.atom.emis_opac(self.T, pops)

    def formal_solve_mali(self, chi, eta):
        shape = (chi.shape[0], self.plan.nz, self.plan.nx)
        _, J_eff, alo_c = self.plan.formal_solve_mali(chi.reshape(shape).contiguous(),
                                                      eta.reshape(shape).contiguous())
        return J_eff, alo_c

    def line_integrals(self, J_eff, alo_c, begin):
        return self.atom.line_integrals(self.T, J_eff, alo_c, begin)

    def stat_eq_integrals(self, integrals, pops):
        return self.atom.stat_eq_integrals(self.T, self.ne, self.n_atom, integrals, pops)


def nlte_solve_sharded(ops, n_lambda: int, pops, tol: float = 1e-3, max_iter: int = 500,
                       group=None):
    """Iterates pops (in place) to a maximum relative change below tol, this rank solving its
    share of the wavelengths.  group: a torch.distributed process group (None: the default
    group if one is initialised, else a single process).  Returns (converged, iterations,
    history); every rank returns the same."""
    import torch.distributed as dist
    use_dist = dist.is_available() and dist.is_initialized()
    rank = dist.get_rank(group) if use_dist else 0
    world = dist.get_world_size(group) if use_dist else 1
    begin, count = lambda_range(rank, world, n_lambda)
    history = []
    for _ in range(max_iter):
        chi, eta = ops.emis_opac(pops)
        J_eff, alo_c = ops.formal_solve_mali(chi[begin:begin + count], eta[begin:begin + count])
        integrals = ops.line_integrals(J_eff, alo_c, begin)
        if world > 1:
            dist.all_reduce(integrals, op=dist.ReduceOp.SUM, group=group)
        dmax = ops.stat_eq_integrals(integrals, pops)
        history.append(dmax)
        if dmax < tol:
            return True, len(history), history
    return False, len(history), history
