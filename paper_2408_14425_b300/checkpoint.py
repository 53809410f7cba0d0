"""Checkpoint and resume of the non-LTE iteration.

The statistical equilibrium keeps no state between iterations besides the populations, so a
checkpoint is the FP64 populations, the number of iterations done, the convergence history
and (optionally) the surrogate's parameters and input normalisation; resuming is passing the
saved populations back to `rcx.nlte_solve`.  Files are numpy .npz archives.
"""
from __future__ import annotations

import numpy as np


def save(path: str, pops, iterations: int, history=(), net=None) -> None:
    """Writes pops ([n_levels][ncell] FP64, device tensor or array), the iteration count, the
    history of maximum relative changes and, with `net`, the MLP parameters (FP32 master
    weights) and normalisation."""
    arrays = {"pops": np.asarray(pops.detach().cpu() if hasattr(pops, "detach") else pops,
                                 dtype=np.float64),
              "iterations": np.int64(iterations),
              "history": np.asarray(list(history), dtype=np.float64)}
    if net is not None:
        theta, mean, std = net.get_params()
        arrays.update(theta=np.asarray(theta, np.float32), mean=np.asarray(mean, np.float32),
                      std=np.asarray(std, np.float32))
    with open(path, "wb") as f:
        np.savez(f, **arrays)


def load(path: str, device=None, net=None):
    """Returns (pops, iterations, history); pops on `device` (a torch device) if given, else
    a numpy array.  With `net`, the saved parameters are loaded into it."""
    with np.load(path) as z:
        pops = z["pops"].copy()
        iterations = int(z["iterations"])
        history = list(z["history"])
        if net is not None:
            if "theta" not in z:
                raise KeyError(f"{path} holds no network parameters")
            net.set_params(z["theta"], z["mean"], z["std"])
    if device is not None:
        import torch
        pops = torch.from_numpy(pops).to(device)
    return pops, iterations, history
