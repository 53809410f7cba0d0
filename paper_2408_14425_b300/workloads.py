"""Seeded synthetic inputs for the radiance-cascade solver.

This module holds input generators only -- none of the method's arithmetic.
It serves both the CUDA path and the FP64 oracle, which import nothing from
each other.  Every generator is deterministic in its seed and returns numpy
arrays laid out [n_lambda][nz][nx] (x fastest).

Recipes (the paper's own MHD snapshot is not available, so these synthetic
fields stand in for it):

* ``disc_field``: 64x64 unit voxels, background chi = 1e-2, eta = 0; a central
  disc of radius 8 voxels (cells whose centre lies within the radius) with
  chi = 1, eta = 1 (source function 1).
* ``grf_fields``: per wavelength two independent 2D Gaussian random fields
  with a k^-5/3 power spectrum (white noise -> FFT -> amplitude |k|^-5/6,
  k = 0 removed -> inverse FFT), each min-max mapped: log10 chi to [-6, 2]
  and log10 S to [-1, 1]; eta = S chi.  Seeds 1000 + l (chi) and 2000 + l (S)
  for wavelength l of a single domain; ``seed_base`` offsets both for the
  batched multi-domain workload.
* ``opaque_disc_field`` / ``thin_disc_field``: the circle tests of Sec. 2.5 and
  the optically thin disc with a closed-form J.
"""
from __future__ import annotations

import functools
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import scipy.fft as _fft


def disc_field(n: int = 64, radius: float = 8.0, chi_bg: float = 1e-2,
               chi_disc: float = 1.0, eta_disc: float = 1.0):
    """Disc of radius `radius` (cell centres inside) in a weakly absorbing background."""
    c = n / 2.0
    x = np.arange(n) + 0.5
    X, Z = np.meshgrid(x, x)
    inside = (X - c) ** 2 + (Z - c) ** 2 <= radius ** 2
    chi = np.full((n, n), chi_bg, dtype=np.float64)
    eta = np.zeros((n, n), dtype=np.float64)
    chi[inside] = chi_disc
    eta[inside] = eta_disc
    return chi[None].astype(np.float32), eta[None].astype(np.float32)


def opaque_disc_field(n: int, radius: float, chi_disc: float = 1e2, source: float = 1.0):
    """Opaque emissive disc in vacuum (cells whose centre is inside; Sec. 2.5 circle test)."""
    c = n / 2.0
    x = np.arange(n) + 0.5
    X, Z = np.meshgrid(x, x)
    inside = (X - c) ** 2 + (Z - c) ** 2 <= radius ** 2
    chi = np.zeros((n, n))
    eta = np.zeros((n, n))
    chi[inside] = chi_disc
    eta[inside] = chi_disc * source
    return chi, eta


def thin_disc_field(n: int, radius: float, chi_disc: float = 1e-9, eta_disc: float = 1.0,
                    supersample: int = 16):
    """Optically thin emitting disc in vacuum with per-cell area coverage (anti-aliased)."""
    c = n / 2.0
    s = supersample
    sub = (np.arange(n * s) + 0.5) / s
    X, Z = np.meshgrid(sub, sub)
    inside = ((X - c) ** 2 + (Z - c) ** 2 <= radius ** 2).astype(np.float64)
    cov = inside.reshape(n, s, n, s).mean(axis=(1, 3))
    chi = chi_disc * cov
    eta = eta_disc * cov
    return chi, eta


@functools.lru_cache(maxsize=8)
def _spectral_amplitude(nx: int, nz: int, slope: float) -> np.ndarray:
    kx = np.fft.rfftfreq(nx)
    kz = np.fft.fftfreq(nz)
    k = np.sqrt(kx[None, :] ** 2 + kz[:, None] ** 2)
    amp = np.zeros_like(k)
    nzk = k > 0
    amp[nzk] = k[nzk] ** (slope / 2.0)
    return amp


def grf(nx: int, nz: int, seed: int, slope: float = -5.0 / 3.0) -> np.ndarray:
    """Zero-mean 2D Gaussian random field with power spectrum ~ |k|^slope."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((nz, nx))
    F = _fft.rfft2(w)
    return _fft.irfft2(F * _spectral_amplitude(nx, nz, slope), s=(nz, nx))


def _minmax(g: np.ndarray, lo: float, hi: float) -> np.ndarray:
    gmin = g.min()
    gmax = g.max()
    return lo + (hi - lo) * (g - gmin) / (gmax - gmin)


def grf_slab(nx: int, nz: int, lam: int, seed_base: int = 0,
             log_chi=(-6.0, 2.0), log_s=(-1.0, 1.0)):
    """(chi, eta) FP64 [nz][nx] of wavelength `lam` of the GRF recipe."""
    lc = _minmax(grf(nx, nz, seed_base + 1000 + lam), *log_chi)
    ls = _minmax(grf(nx, nz, seed_base + 2000 + lam), *log_s)
    chi = 10.0 ** lc
    eta = (10.0 ** ls) * chi
    return chi, eta


def grf_fields(n: int, n_lambda: int, nz: int | None = None, seed_base: int = 0,
               lambdas=None, dtype=np.float32):
    """GRF recipe, all (or the listed) wavelengths: chi, eta [n_l][nz][nx]."""
    nx = n
    nz = n if nz is None else nz
    lams = list(range(n_lambda)) if lambdas is None else list(lambdas)
    chi = np.empty((len(lams), nz, nx), dtype=dtype)
    eta = np.empty((len(lams), nz, nx), dtype=dtype)

    def one(j):
        c, e = grf_slab(nx, nz, lams[j], seed_base)
        chi[j] = c
        eta[j] = e

    workers = max(1, min(len(lams), os.cpu_count() or 1, 16))
    if workers == 1:
        for j in range(len(lams)):
            one(j)
    else:
        with ThreadPoolExecutor(workers) as ex:
            list(ex.map(one, range(len(lams))))
    return chi, eta


def batched_domains(n_domains: int = 16, seed: int = 7, side_min: int = 256,
                    side_max: int = 2048, side_step: int = 64, nl_min: int = 32,
                    nl_max: int = 128):
    """Sizes of the uneven multi-domain workload: list of (side, n_lambda, seed_base)."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_min // side_step, side_max // side_step + 1, size=n_domains) * side_step
    nls = rng.integers(nl_min, nl_max + 1, size=n_domains)
    return [(int(s), int(l), 100_000 * (d + 1)) for d, (s, l) in enumerate(zip(sides, nls))]


# ---------------------------------------------------------------------------
# non-LTE workload: a synthetic 3-level hydrogen-like atom in a prominence slab
# ---------------------------------------------------------------------------

def h3_atom():
    """The synthetic 3-level H-like atom (data only): level energies (eV), statistical
    weights g = 2 n^2, the three lines (lower, upper, A_ul in s^-1), wavelengths per line,
    the frequency-grid half-width in Doppler units at the reference temperature, and the
    atomic mass in amu."""
    return {
        "E_eV": [0.0, 10.2, 12.09],
        "g": [2.0, 8.0, 18.0],
        "lines": [(0, 1, 4.7e8), (0, 2, 5.6e7), (1, 2, 4.4e7)],
        "n_per_line": 21,
        "x_max": 5.0,
        "T_ref": 1.0e4,
        "mass_amu": 1.00794,
    }


def _grf1d(n: int, seed: int, slope: float = -5.0 / 3.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(n)
    F = np.fft.rfft(w)
    k = np.fft.rfftfreq(n)
    amp = np.zeros_like(k)
    amp[k > 0] = k[k > 0] ** (slope / 2.0)
    g = np.fft.irfft(F * amp, n=n)
    return g / g.std()


def prominence_slab(n: int = 512, seed: int = 11, half_width: float = 48.0,
                    blend: float = 8.0, T_cool: float = 6.0e3, T_hot: float = 1.0e6,
                    nH_cool: float = 1.0e18, nH_lo: float = 1.0e15, nH_hi: float = 1.0e18,
                    wander: float = 12.0, voxel_m: float = 5.7e3):
    """Vertical cool dense sheet in a hot corona on an n x n grid of 5.7 km voxels.

    The sheet's centreline x_c(z) = n/2 + wander * g(z), g a unit-variance 1D GRF (k^-5/3);
    log T blends from log T_cool inside to log T_hot outside with tanh((d - half_width) /
    blend), d = |x - x_c(z)|; n_H = nH_cool T_cool / T (constant pressure) times
    10^(0.3 G), G a unit-variance 2D GRF, clipped to [nH_lo, nH_hi].
    Returns T [K], n_H [m^-3] as float64 [n][n] and the voxel size in metres."""
    z = np.arange(n)
    xc = n / 2.0 + wander * _grf1d(n, seed)
    x = np.arange(n) + 0.5
    d = np.abs(x[None, :] - xc[:, None])
    s = 0.5 * (1.0 + np.tanh((d - half_width) / blend))
    logT = np.log10(T_cool) + (np.log10(T_hot) - np.log10(T_cool)) * s
    T = 10.0 ** logT
    G = grf(n, n, seed + 1)
    G = G / G.std()
    nH = np.clip(nH_cool * T_cool / T * 10.0 ** (0.3 * G), nH_lo, nH_hi)
    del z
    return T, nH, voxel_m
