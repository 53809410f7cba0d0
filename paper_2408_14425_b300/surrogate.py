"""Orchestration of the surrogate-seeded non-LTE solve (calls into librcx.so only).

Every numerical step runs in the library's kernels: LTE start, opacity/emissivity,
the formal solution, the network's forward pass and training, and the statistical
equilibrium.  This module strings the calls together:

* ``first_J`` -- the formal solution at the LTE populations (the first iteration's J),
  whose line-centre values are three of the network's six features;
* ``training_pairs`` -- features at LTE and log departure coefficients of the converged
  populations of one atmosphere;
* ``solve`` -- the iteration from LTE (``net=None``) or from the network's seed, timed;
* ``train_stepped`` -- Adam through the library with the learning rate halved over equal
  segments.
"""
from __future__ import annotations

import time

from . import rcx


def first_J(plan, atom, T, pops, stream=None):
    import torch
    chi, eta = atom.emis_opac(T, pops, stream=stream)
    nl = atom.n_lambda
    shape = (nl, plan.nz, plan.nx)
    J = torch.empty(shape, dtype=torch.float32, device=T.device)
    J_eff = torch.empty_like(J)
    alo_c = torch.empty_like(J)
    plan.formal_solve_mali(chi.reshape(shape), eta.reshape(shape), J=J, J_eff=J_eff, alo_c=alo_c,
                           stream=stream)
    return J


def training_pairs(plan, atom, T, nH, tol=1e-3, max_iter=1000):
    """(X [ncell][6], Y [ncell][3], iterations) for one atmosphere."""
    ne, na, pops = atom.lte(T, nH)
    X = rcx.surrogate_features(atom, T, ne, nH, first_J(plan, atom, T, pops))
    conv, it, _ = rcx.nlte_solve(plan, atom, T, ne, na, pops, tol=tol, max_iter=max_iter)
    if not conv:
        raise RuntimeError(f"training atmosphere did not converge in {max_iter} iterations")
    return X, rcx.surrogate_targets(atom, T, na, pops), it


def solve(plan, atom, T, nH, net=None, tol=1e-3, max_iter=2000):
    """Non-LTE solve from LTE or from the network's seed; wall time includes the seed
    (features' formal solution, forward pass) and every iteration.
    Returns dict(pops, converged, iterations, seconds, history, fallback)."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ne, na, pops = atom.lte(T, nH)
    fallback = 0
    if net is not None:
        X = rcx.surrogate_features(atom, T, ne, nH, first_J(plan, atom, T, pops))
        fallback = rcx.surrogate_seed(atom, net, X, T, na, pops)
    conv, it, hist = rcx.nlte_solve(plan, atom, T, ne, na, pops, tol=tol, max_iter=max_iter)
    torch.cuda.synchronize()
    return dict(pops=pops, converged=conv, iterations=it, seconds=time.perf_counter() - t0,
                history=hist, fallback=fallback, ne=ne, n_atom=na)


def train_stepped(net, X, Y, steps: int, batch: int = 4096, lr0: float = 4e-3, segments: int = 4):
    """Adam (the library's kernels) for `steps` minibatch steps in `segments` equal parts, the
    learning rate halved from one part to the next (lr0, lr0/2, ...).  Returns the recorded
    minibatch losses."""
    hist = []
    per = max(1, steps // segments)
    done = 0
    for k in range(segments):
        n = per if k < segments - 1 else steps - done
        if n <= 0:
            break
        hist += net.train(X, Y, batch=batch, steps=n, lr=lr0 * 0.5 ** k)
        done += n
    return hist
