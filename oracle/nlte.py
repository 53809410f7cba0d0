"""FP64 oracle of the non-LTE population update driven by the RC formal solution.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline timing).  Plain numpy,
vectorised over cells, in the order of Sec. 3.3 of the paper:

  1. opacity and emissivity of every line wavelength from the populations
     (RTE of Sec. 3.2, Eq. 15-16 need chi and eta);
  2. the formal solution gives J and the diagonal operator Lambda* (Eq. 17,
     read as 1 - exp(-tau_centre->edge));
  3. MALI rates with "same preconditioning" (Sec. 3.3): the effective
     intensity of each transition is I_eff = I_dagger - Psi* U (Eq. 18-19),
     Psi* = Lambda*/chi; only the off-diagonal rates are accumulated and the
     diagonal follows from conservation;
  4. Gamma n = 0 (Eq. 20) per cell, solved in FP64 with one row replaced by
     particle conservation;
  5. convergence: the maximum relative population change (Sec. 4.2, 1e-3).

Readings of what the paper leaves open (also listed in the design notes):
  * Rates (Rybicki & Hummer 1992 in same-preconditioning form, diagonal ALO).  With
    hnu/4pi folded away, per line and cell
        Jbar = sum_k w_k phi_k J_k,   Lbar = sum_k w_k phi_k Lambda*_k,
        R_lu = B_lu (Jbar - S_dagger Lbar),
        R_ul = A_ul (1 - Lbar) + B_ul (Jbar - S_dagger Lbar),
    S_dagger the line source function at the previous populations (constant over the
    line because B and h nu are taken at line centre).  Lambda* = 0 gives plain
    Lambda iteration.
  * Gaussian profiles, 21 frequencies uniform in Doppler units at T_ref on +-x_max,
    trapezoid weights in frequency; the profile is renormalised per cell so that
    sum_k w_k phi_k = 1 (keeps detailed balance exact on the discrete grid).
  * Collisions: van Regemorter (1962) collision strength
        Omega_lu = (8 pi / sqrt 3) (E_Ryd / dE) g_l f_lu P(y),
        P(y) = max(0.2, 0.276 e^y E1(y)),  y = dE/kT,
    turned into a rate with the textbook relation
        C_lu = n_e beta Omega_lu / (g_l sqrt T) e^-y,   beta = h^2 / ((2 pi m_e)^1.5 k^0.5),
    and C_ul from detailed balance.
  * n_e and the neutral density n_atom from LTE Saha ionisation of pure hydrogen at
    (T, n_H), held fixed (no charge conservation).
  * The conservation row replaces the equation of the most populated level of the
    previous iterate.
  * Intensities in SI per unit frequency (W m^-2 Hz^-1 sr^-1), chi in m^-1.
"""
from __future__ import annotations

import numpy as np
from scipy import special

# CODATA 2018
H = 6.62607015e-34
C = 2.99792458e8
KB = 1.380649e-23
EV = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
QE = 1.602176634e-19
EPS0 = 8.8541878128e-12
E_RYD = 13.605693122994 * EV      # Rydberg energy (van Regemorter's E_H)
CHI_H = 13.598434599702 * EV      # hydrogen ionisation energy


# ---------------------------------------------------------------------------
# atom
# ---------------------------------------------------------------------------

def line_constants(atom):
    """Per line: nu0, B_ul, B_lu (intensity per unit frequency), f_lu, dE."""
    E = np.asarray(atom["E_eV"], dtype=np.float64) * EV
    g = np.asarray(atom["g"], dtype=np.float64)
    out = []
    for lo, up, A in atom["lines"]:
        dE = E[up] - E[lo]
        nu0 = dE / H
        Bul = A * C ** 2 / (2.0 * H * nu0 ** 3)
        Blu = g[up] / g[lo] * Bul
        f_lu = A * EPS0 * ME * C ** 3 * g[up] / (2.0 * np.pi * QE ** 2 * nu0 ** 2 * g[lo])
        out.append(dict(lo=lo, up=up, A=A, nu0=nu0, Bul=Bul, Blu=Blu, f_lu=f_lu, dE=dE))
    return out


def frequency_grid(atom):
    """Per line: frequencies nu_k and trapezoid weights w_k (Hz) of the fixed grid."""
    m = atom["mass_amu"] * AMU
    n = atom["n_per_line"]
    x = np.linspace(-atom["x_max"], atom["x_max"], n)
    grids = []
    for L in line_constants(atom):
        dnu_ref = L["nu0"] / C * np.sqrt(2.0 * KB * atom["T_ref"] / m)
        nu = L["nu0"] + x * dnu_ref
        w = np.full(n, nu[1] - nu[0])
        w[0] *= 0.5
        w[-1] *= 0.5
        grids.append((nu, w))
    return grids


def profiles(atom, T):
    """phi[line][k][cell]: Gaussian at the local Doppler width, renormalised so that
    sum_k w_k phi_k = 1 in every cell."""
    T = np.asarray(T, dtype=np.float64).ravel()
    m = atom["mass_amu"] * AMU
    out = []
    for L, (nu, w) in zip(line_constants(atom), frequency_grid(atom)):
        dnu = L["nu0"] / C * np.sqrt(2.0 * KB * T / m)               # [cell]
        u = (nu[:, None] - L["nu0"]) / dnu[None, :]
        phi = np.exp(-u * u) / (np.sqrt(np.pi) * dnu[None, :])
        phi = phi / np.sum(w[:, None] * phi, axis=0, keepdims=True)
        out.append(phi)
    return out


def planck_nu(nu, T):
    """Planck function B_nu(T) in W m^-2 Hz^-1 sr^-1."""
    return 2.0 * H * nu ** 3 / C ** 2 / np.expm1(H * nu / (KB * np.asarray(T, dtype=np.float64)))


# ---------------------------------------------------------------------------
# LTE
# ---------------------------------------------------------------------------

def saha_hydrogen(T, nH):
    """Pure-hydrogen LTE ionisation: returns (n_e, n_neutral).
    n_e n_p / n_HI = (2 pi m_e k T / h^2)^1.5 exp(-chi_H / kT)  (U_HI = 2, U_HII = 1)."""
    T = np.asarray(T, dtype=np.float64)
    nH = np.asarray(nH, dtype=np.float64)
    phi = (2.0 * np.pi * ME * KB * T / H ** 2) ** 1.5 * np.exp(-CHI_H / (KB * T))
    s = np.sqrt(phi * phi + 4.0 * nH * phi)
    x = 2.0 * phi / (phi + s)                                        # x^2 nH / (1 - x) = phi
    ne = x * nH
    n_atom = nH * (4.0 * nH * phi / (phi + s) ** 2)                  # nH (1 - x), no cancellation
    return ne, n_atom


def lte_populations(atom, T, n_atom):
    """Boltzmann distribution over the model's levels, normalised to n_atom: [level][cell]."""
    T = np.asarray(T, dtype=np.float64).ravel()
    n_atom = np.asarray(n_atom, dtype=np.float64).ravel()
    E = np.asarray(atom["E_eV"], dtype=np.float64) * EV
    g = np.asarray(atom["g"], dtype=np.float64)
    b = g[:, None] * np.exp(-E[:, None] / (KB * T[None, :]))
    return n_atom[None, :] * b / b.sum(axis=0, keepdims=True)


# ---------------------------------------------------------------------------
# opacity / emissivity (from populations)
# ---------------------------------------------------------------------------

def emis_opac(atom, T, pops):
    """chi [m^-1], eta [W m^-3 Hz^-1 sr^-1] of every grid frequency: [line*n_per_line][cell].
    chi = (h nu0 / 4 pi)(n_l B_lu - n_u B_ul) phi,  eta = (h nu0 / 4 pi) n_u A_ul phi."""
    pops = np.asarray(pops, dtype=np.float64)
    phis = profiles(atom, T)
    chi, eta = [], []
    for L, phi in zip(line_constants(atom), phis):
        k = H * L["nu0"] / (4.0 * np.pi)
        nl, nu_ = pops[L["lo"]], pops[L["up"]]
        chi.append(k * (nl * L["Blu"] - nu_ * L["Bul"])[None, :] * phi)
        eta.append(k * (nu_ * L["A"])[None, :] * phi)
    return np.concatenate(chi, axis=0), np.concatenate(eta, axis=0)


def line_source_function(atom, pops):
    """S per line and cell: n_u A / (n_l B_lu - n_u B_ul)."""
    pops = np.asarray(pops, dtype=np.float64)
    return [pops[L["up"]] * L["A"] / (pops[L["lo"]] * L["Blu"] - pops[L["up"]] * L["Bul"])
            for L in line_constants(atom)]


# ---------------------------------------------------------------------------
# collisions
# ---------------------------------------------------------------------------

BETA_COLL = H ** 2 / ((2.0 * np.pi * ME) ** 1.5 * np.sqrt(KB))      # m^3 s^-1 K^0.5


def van_regemorter_P(y):
    y = np.asarray(y, dtype=np.float64)
    return np.maximum(0.2, 0.276 * special.exp1(y) * np.exp(y))


def collision_rates(atom, T, ne):
    """(C_lu, C_ul) per line and cell [s^-1] (van Regemorter 1962 + detailed balance)."""
    T = np.asarray(T, dtype=np.float64).ravel()
    ne = np.asarray(ne, dtype=np.float64).ravel()
    g = np.asarray(atom["g"], dtype=np.float64)
    out = []
    for L in line_constants(atom):
        y = L["dE"] / (KB * T)
        omega = (8.0 * np.pi / np.sqrt(3.0)) * (E_RYD / L["dE"]) * g[L["lo"]] * L["f_lu"] \
            * van_regemorter_P(y)
        Clu = ne * BETA_COLL * omega / (g[L["lo"]] * np.sqrt(T)) * np.exp(-y)
        Cul = Clu * g[L["lo"]] / g[L["up"]] * np.exp(y)
        out.append((Clu, Cul))
    return out


# ---------------------------------------------------------------------------
# statistical equilibrium (Sec. 3.3, Eq. 18-20)
# ---------------------------------------------------------------------------

def effective_inputs(atom, J, alo, pops_old):
    """(J_eff, 1 - Lambda*) per wavelength: J_eff = J - Lambda* S_dagger (Eq. 19 with a
    diagonal operator; Psi* eta_dagger = Lambda* S_dagger)."""
    npl = atom["n_per_line"]
    J = np.asarray(J, dtype=np.float64)
    alo = np.zeros_like(J) if alo is None else np.asarray(alo, dtype=np.float64).reshape(J.shape)
    S_old = line_source_function(atom, pops_old)
    Jeff = np.empty_like(J)
    for li, S in enumerate(S_old):
        sl = slice(li * npl, (li + 1) * npl)
        Jeff[sl] = J[sl] - S[None, :] * alo[sl]
    return Jeff, 1.0 - alo


def line_integrals(atom, T, J_eff, alo_c, lambda_begin=0):
    """The two radiation integrals of each line's rates (Sec. 3.3) over the grid wavelengths
    [lambda_begin, lambda_begin + len(J_eff)) (global indices, line after line):
    Jbar = sum_k w phi J_eff and Lbar = sum_k w phi (1 - Lambda*), [line][2][cell], with phi
    normalised over the whole line, so integrals over disjoint ranges add up to the line's.
    alo_c = None means Lambda* = 0."""
    T = np.asarray(T, dtype=np.float64).ravel()
    ncell = T.size
    npl = atom["n_per_line"]
    J_eff = np.asarray(J_eff, dtype=np.float64).reshape(-1, ncell)
    cnt = J_eff.shape[0]
    alo_c = np.ones_like(J_eff) if alo_c is None else \
        np.asarray(alo_c, dtype=np.float64).reshape(-1, ncell)
    phis = profiles(atom, T)
    grids = frequency_grid(atom)
    out = np.zeros((len(phis), 2, ncell))
    for li, (phi, (nu, w)) in enumerate(zip(phis, grids)):
        ks = [k for k in range(npl) if 0 <= li * npl + k - lambda_begin < cnt]
        if not ks:
            continue
        rows = [li * npl + k - lambda_begin for k in ks]
        wphi = w[ks, None] * phi[ks]
        out[li, 0] = np.sum(wphi * J_eff[rows], axis=0)
        out[li, 1] = np.sum(wphi * alo_c[rows], axis=0)
    return out


def rate_matrix_from_integrals(atom, T, ne, integrals):
    """Gamma [cell][i][j] (rate j -> i per atom in j off the diagonal, diagonal from
    conservation) from each line's Jbar and Lbar [line][2][cell]:
    R_lu = B_lu Jbar, R_ul = A_ul Lbar + B_ul Jbar, plus the collisions."""
    T = np.asarray(T, dtype=np.float64).ravel()
    ncell = T.size
    nlev = len(atom["E_eV"])
    integrals = np.asarray(integrals, dtype=np.float64).reshape(-1, 2, ncell)
    coll = collision_rates(atom, T, ne)
    G = np.zeros((ncell, nlev, nlev))
    for li, (L, (Clu, Cul)) in enumerate(zip(line_constants(atom), coll)):
        Jb, Lc = integrals[li, 0], integrals[li, 1]
        Rlu = L["Blu"] * Jb
        Rul = L["A"] * Lc + L["Bul"] * Jb
        G[:, L["up"], L["lo"]] += Rlu + Clu
        G[:, L["lo"], L["up"]] += Rul + Cul
    for i in range(nlev):
        G[:, i, i] = -np.sum(G[:, :, i], axis=1)
    return G


def rate_matrix_eff(atom, T, ne, J_eff, alo_c):
    """Gamma [cell][i][j] from the effective intensity: rate j -> i per atom in j
    (off-diagonal), diagonal from conservation.  J_eff, alo_c: [line*n_per_line][cell];
    alo_c = None means Lambda* = 0."""
    return rate_matrix_from_integrals(atom, T, ne, line_integrals(atom, T, J_eff, alo_c))


def rate_matrix(atom, T, ne, J, alo, pops_old):
    """Gamma from J and Lambda* (MALI, same preconditioning, diagonal operator)."""
    ncell = np.asarray(T).size
    J = np.asarray(J, dtype=np.float64).reshape(-1, ncell)
    Jeff, aloc = effective_inputs(atom, J, alo, pops_old)
    return rate_matrix_eff(atom, T, ne, Jeff, aloc)


def solve_populations(G, n_atom, pops_old):
    """Gamma n = 0 with the most populated level's row replaced by sum n = n_atom."""
    G = np.array(G, dtype=np.float64, copy=True)
    ncell, nlev, _ = G.shape
    n_atom = np.asarray(n_atom, dtype=np.float64).ravel()
    r = np.argmax(np.asarray(pops_old).reshape(nlev, ncell), axis=0)
    b = np.zeros((ncell, nlev))
    G[np.arange(ncell), r, :] = 1.0
    b[np.arange(ncell), r] = n_atom
    return np.linalg.solve(G, b[..., None])[..., 0].T                  # [level][cell]


def stat_eq(atom, T, ne, n_atom, J, alo, pops_old):
    """New populations and the maximum relative change max |n_new - n_old| / n_new."""
    G = rate_matrix(atom, T, ne, J, alo, pops_old)
    new = solve_populations(G, n_atom, pops_old)
    old = np.asarray(pops_old, dtype=np.float64).reshape(new.shape)
    rel = np.abs(new - old) / np.abs(new)
    return new, float(np.max(rel))


def stat_eq_integrals(atom, T, ne, n_atom, integrals, pops_old):
    """stat_eq from each line's radiation integrals summed over all its wavelengths."""
    G = rate_matrix_from_integrals(atom, T, ne, integrals)
    new = solve_populations(G, n_atom, pops_old)
    old = np.asarray(pops_old, dtype=np.float64).reshape(new.shape)
    rel = np.abs(new - old) / np.abs(new)
    return new, float(np.max(rel))


def stat_eq_eff(atom, T, ne, n_atom, J_eff, alo_c, pops_old):
    """stat_eq from (J_eff, 1 - Lambda*) directly."""
    G = rate_matrix_eff(atom, T, ne, J_eff, alo_c)
    new = solve_populations(G, n_atom, pops_old)
    old = np.asarray(pops_old, dtype=np.float64).reshape(new.shape)
    rel = np.abs(new - old) / np.abs(new)
    return new, float(np.max(rel))


def nlte_iterate(atom, T, nH, voxel_m, n_cascades, max_iter=50, tol=1e-3, pops0=None,
                 callback=None, **rc_kw):
    """The iteration of Sec. 3.3 with the RC oracle as formal solver (small grids only)."""
    from . import rc_solve
    T = np.asarray(T, dtype=np.float64)
    shape = T.shape
    ne, n_atom = saha_hydrogen(T.ravel(), np.asarray(nH, dtype=np.float64).ravel())
    pops = lte_populations(atom, T, n_atom) if pops0 is None else np.array(pops0, dtype=np.float64)
    history = []
    for it in range(max_iter):
        chi, eta = emis_opac(atom, T, pops)
        J, alo, _ = rc_solve(chi.reshape(-1, *shape), eta.reshape(-1, *shape), n_cascades,
                             voxel=voxel_m, want_alo=True, **rc_kw)
        pops, dmax = stat_eq(atom, T, ne, n_atom, J.reshape(chi.shape), alo.reshape(chi.shape),
                             pops)
        history.append(dmax)
        if callback:
            callback(it, pops, J)
        if dmax < tol:
            break
    return pops, history
