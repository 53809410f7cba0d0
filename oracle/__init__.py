"""FP64 CPU oracle of the radiance-cascade formal solution (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never does, and
this package imports nothing from it.  The arithmetic lives in
``rc_oracle.c`` (FP64, OpenMP over probes); this module compiles it with gcc
and wraps it with ctypes and numpy.

Passages followed (details in the C source):
  radiance interval, Eq. 9 (Sec. 2.2); merge operator, Eq. 11 (Sec. 2.2.1);
  scaling law, Eq. 12-13 (Sec. 2.3); bilinear interpolation and child-cone
  averaging (Sec. 2.3.1); edge clamp (Sec. 2.5); piecewise-constant update,
  Eq. 16 (Sec. 3.2); J, Eq. 1; diagonal ALO, Eq. 17 (Sec. 3.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["rc_oracle.c"]
_LIB_PATH = os.path.join(_HERE, "librcoracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_llp = ctypes.POINTER(ctypes.c_longlong)


def _sources():
    return [os.path.join(_HERE, s) for s in _SOURCES]


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (FP64, -O2, OpenMP, no fast-math)."""
    srcs = _sources()
    if not force and os.path.exists(_LIB_PATH):
        lib_m = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= lib_m for s in srcs):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-Wall",
           "-fno-fast-math", *srcs, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.rco_interval.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, _dp, _dp]
        L.rco_probes.argtypes = [ctypes.c_int, ctypes.c_int]
        L.rco_probes.restype = ctypes.c_int
        L.rco_dirs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.rco_dirs.restype = ctypes.c_longlong
        L.rco_direction.argtypes = [ctypes.c_longlong, ctypes.c_longlong, _dp, _dp]
        L.rco_march.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.rco_march.restype = ctypes.c_longlong
        L.rco_merge.argtypes = [ctypes.c_double] * 4 + [_dp, _dp]
        L.rco_rc_solve.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int, _dp, _dp, _llp]
        L.rco_rc_solve.restype = ctypes.c_int
        L.rco_rc_solve_fix.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp, _dp, _llp]
        L.rco_rc_solve_fix.restype = ctypes.c_int
        L.rco_rc_solve_sparse.argtypes = [_dp, _dp, ctypes.c_char_p, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _llp]
        L.rco_rc_solve_sparse.restype = ctypes.c_int
        L.rco_emergent.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, _dp]
        L.rco_emergent.restype = ctypes.c_double
        L.rco_count_crossings.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_int, _llp]
        L.rco_count_crossings.restype = ctypes.c_longlong
        L.rco_lc_solve.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_int, _dp]
        L.rco_lc_solve.restype = ctypes.c_int
        L.rco_num_threads.restype = ctypes.c_int
        L.rco_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def interval(i: int, n_cascades: int, interval0: float = 1.0, branching: int = 4,
             rule: int = 0) -> tuple[float, float]:
    """[a_i, b_i] of cascade i in voxels (Eq. 12-13; top cascade b = inf)."""
    a = ctypes.c_double()
    b = ctypes.c_double()
    lib().rco_interval(rule, interval0, branching, i, n_cascades, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def probes(n: int, i: int) -> int:
    return lib().rco_probes(n, i)


def dirs(dirs0: int, branching: int, i: int) -> int:
    return lib().rco_dirs(dirs0, branching, i)


def direction(k: int, W: int) -> tuple[float, float]:
    wx = ctypes.c_double()
    wz = ctypes.c_double()
    lib().rco_direction(k, W, ctypes.byref(wx), ctypes.byref(wz))
    return wx.value, wz.value


# --------------------------------------------------------------------------
# one interval, merge
# --------------------------------------------------------------------------

def march(chi, eta, origin, omega, a, b, voxel: float = 1.0):
    """R_{a,b}(origin, omega) of one slab: returns (I, tau, crossings)."""
    chi = _f64(chi)
    eta = _f64(eta)
    nz, nx = chi.shape
    I = ctypes.c_double()
    tau = ctypes.c_double()
    n = lib().rco_march(_ptr(chi), _ptr(eta), nx, nz, voxel, float(origin[0]), float(origin[1]),
                        float(omega[0]), float(omega[1]), float(a), float(b),
                        ctypes.byref(I), ctypes.byref(tau))
    return I.value, tau.value, int(n)


def merge(near, far):
    """M(R_near, R_far) for (I, tau) pairs of contiguous intervals (Eq. 11, reading R1)."""
    I = ctypes.c_double()
    tau = ctypes.c_double()
    lib().rco_merge(near[0], near[1], far[0], far[1], ctypes.byref(I), ctypes.byref(tau))
    return I.value, tau.value


# --------------------------------------------------------------------------
# full solves
# --------------------------------------------------------------------------

def rc_solve(chi, eta, n_cascades: int, dirs0: int = 4, branching: int = 4,
             interval0: float = 1.0, rule: int = 0, voxel: float = 1.0,
             want_alo: bool = False, threads: int | None = None, bilinear_fix: bool = False):
    """RC formal solution.  chi/eta: [n_lambda][nz][nx] (or [nz][nx]).

    Returns (J, alo or None, crossings_per_level of one wavelength), J in FP64.
    bilinear_fix selects the bilinear fix of Sec. 2.5.
    """
    chi = _f64(chi)
    eta = _f64(eta)
    squeeze = chi.ndim == 2
    if squeeze:
        chi = chi[None]
        eta = eta[None]
    nl, nz, nx = chi.shape
    J = np.zeros_like(chi)
    alo = np.zeros_like(chi) if want_alo else None
    cross = np.zeros(n_cascades, dtype=np.int64)
    L = lib()
    if threads is not None:
        L.rco_set_num_threads(int(threads))
    rc = L.rco_rc_solve_fix(_ptr(chi), _ptr(eta), nx, nz, nl, voxel, n_cascades, dirs0,
                            branching, interval0, rule, int(bilinear_fix), _ptr(J),
                            _ptr(alo) if alo is not None else None, cross.ctypes.data_as(_llp))
    if rc != 0:
        raise ValueError("rco_rc_solve rejected its arguments")
    if squeeze:
        J = J[0]
        alo = alo[0] if alo is not None else None
    return J, alo, cross


def gauss_radau_inclinations(n: int):
    """n-point Gauss-Radau rule for mu = cos(angle to the invariant y axis) on [0, 1] with
    the fixed node at mu = 0 (the in-plane ray): nodes and weights summing to 1.
    From the rule on [-1, 1] with the fixed node -1: the free nodes are the roots of
    (P_{n-1} + P_n)/(1 + x), weights 2/n^2 at -1 and (1 - x)/(n P_{n-1}(x))^2 elsewhere."""
    from numpy.polynomial import legendre as L
    if n == 1:
        return np.array([0.0]), np.array([1.0])
    c = np.zeros(n + 1)
    c[n - 1] = 1.0
    c[n] = 1.0
    roots = np.sort(np.real(L.legroots(c)))
    roots = roots[np.abs(roots + 1.0) > 1e-10]
    e = np.zeros(n)
    e[n - 1] = 1.0
    x = np.concatenate([[-1.0], roots])
    w = np.concatenate([[2.0 / n ** 2], (1.0 - roots) / (n * L.legval(roots, e)) ** 2])
    return (x + 1.0) / 2.0, w / 2.0


def rc_solve_inclined(chi, eta, n_cascades: int, n_incl: int, want_alo: bool = False, **kw):
    """2D invariance (Sec. 3.1): every flatland ray stands for n_incl rays with the same x-z
    projection and inclinations mu_j to the invariant axis.  Along such a ray the path per
    projected length is 1/sqrt(1 - mu_j^2), so each inclination is the flatland problem with
    chi and eta scaled by that factor; J (and alo) are their Gauss-Radau weighted sum."""
    mu, w = gauss_radau_inclinations(n_incl)
    chi = _f64(chi)
    eta = _f64(eta)
    J = 0.0
    alo = 0.0 if want_alo else None
    for m, wj in zip(mu, w):
        r = 1.0 / np.sqrt(1.0 - m * m)
        Jj, aj, _ = rc_solve(chi * r, eta * r, n_cascades, want_alo=want_alo, **kw)
        J = J + wj * Jj
        if want_alo:
            alo = alo + wj * aj
    return J, alo


def rc_solve_sparse(chi, eta, active, n_cascades: int, dirs0: int = 4, branching: int = 4,
                    interval0: float = 1.0, rule: int = 0, voxel: float = 1.0):
    """Sparse RC of one slab (Sec. 3.5): returns (J, intervals computed per cascade)."""
    chi = _f64(chi)
    eta = _f64(eta)
    nz, nx = chi.shape
    act = np.ascontiguousarray(np.asarray(active, dtype=np.uint8))
    J = np.zeros_like(chi)
    rays = np.zeros(n_cascades, dtype=np.int64)
    rc = lib().rco_rc_solve_sparse(_ptr(chi), _ptr(eta), act.tobytes(), nx, nz, voxel, n_cascades,
                                   dirs0, branching, interval0, rule, _ptr(J),
                                   rays.ctypes.data_as(_llp))
    if rc != 0:
        raise ValueError("rco_rc_solve_sparse rejected its arguments")
    return J, rays


def emergent(chi, eta, rays, voxel: float = 1.0, mu: float = 0.0, want_contrib: bool = False):
    """Front-to-back long characteristics (Sec. 3.9): intensity reaching each ray origin from
    along its direction, rays [n][4] = (ox, oz, wx, wz) in voxel units, for one slab.  mu is
    the inclination to the invariant axis (path per projected length 1/sqrt(1 - mu^2)).
    Returns I [n] and, with want_contrib, the contribution function summed per cell."""
    r = 1.0 / np.sqrt(1.0 - mu * mu)
    chi = _f64(chi) * r
    eta = _f64(eta) * r
    nz, nx = chi.shape
    rays = np.asarray(rays, dtype=np.float64)
    I = np.zeros(len(rays))
    C = np.zeros_like(chi) if want_contrib else None
    L = lib()
    for i, (ox, oz, wx, wz) in enumerate(rays):
        I[i] = L.rco_emergent(_ptr(chi), _ptr(eta), nx, nz, voxel, ox, oz, wx, wz,
                              _ptr(C) if C is not None else None)
    return (I, C) if want_contrib else I


def count_crossings(nx: int, nz: int, n_cascades: int, dirs0: int = 4, branching: int = 4,
                    interval0: float = 1.0, rule: int = 0):
    """Voxel crossings per cascade of one wavelength (geometry only)."""
    per = np.zeros(n_cascades, dtype=np.int64)
    tot = lib().rco_count_crossings(nx, nz, n_cascades, dirs0, branching, interval0, rule,
                                    per.ctypes.data_as(_llp))
    return int(tot), per


def lc_solve(chi, eta, n_angles: int, voxel: float = 1.0):
    """Brute-force long-characteristics J of one slab (n_angles in-plane rays per cell)."""
    chi = _f64(chi)
    eta = _f64(eta)
    nz, nx = chi.shape
    J = np.zeros_like(chi)
    rc = lib().rco_lc_solve(_ptr(chi), _ptr(eta), nx, nz, voxel, n_angles, _ptr(J))
    if rc != 0:
        raise ValueError("rco_lc_solve rejected its arguments")
    return J


def num_threads() -> int:
    return lib().rco_num_threads()
