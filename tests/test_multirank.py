"""The multi-GPU path of the benchmark on CPU: two gloo ranks get disjoint wavelength
batches of independent problems, and the step time reported is the slowest rank's."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2408_14425_b300 import workloads
    lams = bench.rank_lambdas(rank, 4)
    chi, _ = workloads.grf_fields(32, 4, lambdas=lams)
    t = bench.max_over_ranks(10.0 + rank, dist)
    dist.barrier()
    out[rank] = (lams, float(chi.sum()), t)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_wavelengths_and_take_the_max_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    l0, s0, t0 = res[0]
    l1, s1, t1 = res[1]
    assert l0 == [0, 1, 2, 3] and l1 == [4, 5, 6, 7]
    assert not set(l0) & set(l1)
    assert s0 != s1                      # independent fields per rank
    assert t0 == t1 == 11.0              # the slowest rank's time on every rank


def test_single_rank_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.rank_lambdas(0, 64) == list(range(64))


class _OracleOps:
    """The four steps of a non-LTE iteration through the FP64 oracle (CPU), with the line
    integrals as torch CPU tensors so that gloo can all-reduce them."""

    def __init__(self, atom, T, nH, vox, n_cascades):
        from oracle import nlte
        self.nlte, self.atom, self.T, self.vox, self.C = nlte, atom, T, vox, n_cascades
        self.ne, self.n_atom = nlte.saha_hydrogen(T.ravel(), nH.ravel())

    def emis_opac(self, pops):
        return self.nlte.emis_opac(self.atom, self.T, pops)

    def formal_solve_mali(self, chi, eta):
        import oracle
        shape = (chi.shape[0],) + self.T.shape
        J, alo, _ = oracle.rc_solve(chi.reshape(shape), eta.reshape(shape), self.C,
                                    voxel=self.vox, want_alo=True)
        return J.reshape(chi.shape), alo.reshape(chi.shape)

    def line_integrals(self, J, alo, begin):
        # MALI inputs from J and Lambda* (Eq. 19 with a diagonal operator)
        pops = self._pops
        npl = self.atom["n_per_line"]
        S = self.nlte.line_source_function(self.atom, pops)
        lam = np.arange(begin, begin + J.shape[0])
        J_eff = J - np.stack([S[l // npl] for l in lam]) * alo
        out = self.nlte.line_integrals(self.atom, self.T, J_eff, 1.0 - alo, begin)
        return torch.from_numpy(out)

    def stat_eq_integrals(self, integrals, pops):
        new, d = self.nlte.stat_eq_integrals(self.atom, self.T, self.ne, self.n_atom,
                                             integrals.numpy(), pops)
        pops[...] = new
        return d


class _OracleOpsKeep(_OracleOps):
    def emis_opac(self, pops):
        self._pops = pops.copy()
        return super().emis_opac(pops)


def _nlte_case():
    from paper_2408_14425_b300 import workloads as W
    T, nH, vox = W.prominence_slab(n=16, half_width=3.2, blend=2, wander=1, nH_cool=1e17,
                                   nH_lo=1e14, nH_hi=1e17)
    return W.h3_atom(), T, nH, vox


def _sharded_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import nlte
    from paper_2408_14425_b300 import distributed
    atom, T, nH, vox = _nlte_case()
    ops = _OracleOpsKeep(atom, T, nH, vox, 4)
    pops = nlte.lte_populations(atom, T, ops.n_atom)
    conv, it, hist = distributed.nlte_solve_sharded(ops, 63, pops, tol=1e-30, max_iter=4)
    out[rank] = (pops.copy(), hist, distributed.lambda_range(rank, world, 63))
    dist.destroy_process_group()


def test_wavelength_split_nlte_over_two_gloo_ranks_equals_one_rank():
    """Two gloo ranks each solve half of the 63 line wavelengths, all-reduce the per-line
    radiation integrals (6 FP64 per cell) and update the populations: after 4 iterations
    both hold the populations of the unsplit iteration to 1e-12, and the same history."""
    from oracle import nlte
    from paper_2408_14425_b300 import distributed
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_sharded_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    atom, T, nH, vox = _nlte_case()
    ops = _OracleOpsKeep(atom, T, nH, vox, 4)
    pops = nlte.lte_populations(atom, T, ops.n_atom)
    conv, it, hist = distributed.nlte_solve_sharded(ops, 63, pops, tol=1e-30, max_iter=4)
    assert res[0][2] == (0, 32) and res[1][2] == (32, 31)
    for r in range(world):
        np.testing.assert_allclose(res[r][0], pops, rtol=1e-12)
        np.testing.assert_allclose(res[r][1], hist, rtol=1e-9)
    np.testing.assert_array_equal(res[0][0], res[1][0])     # identical on every rank


def test_lambda_range_partitions_the_wavelengths():
    from paper_2408_14425_b300 import distributed
    for n, world in [(63, 2), (63, 4), (64, 8), (5, 5)]:
        got = [distributed.lambda_range(r, world, n) for r in range(world)]
        assert sum(c for _, c in got) == n
        assert [b for b, _ in got] == [sum(c for _, c in got[:r]) for r in range(world)]
        assert max(c for _, c in got) - min(c for _, c in got) <= 1


def test_batched_domains_are_dealt_out_by_cost():
    """The batched workload over N ranks: every domain goes to exactly one rank, and the
    largest rank's cost (side^2 x wavelengths) is within the largest single domain of the
    mean (greedy largest-first assignment)."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2408_14425_b300 import workloads
    doms = workloads.batched_domains()
    cost = [s * s * nl for s, nl, _ in doms]
    for world in (1, 2, 4, 8):
        parts = [bench.rank_domains(r, world, doms) for r in range(world)]
        flat = sorted(d for p in parts for d in p)
        assert flat == list(range(len(doms)))
        loads = [sum(cost[d] for d in p) for p in parts]
        assert max(loads) - sum(loads) / world <= max(cost)
    assert bench.rank_domains(0, 1, doms) == list(range(len(doms)))
