"""Pins of the FP64 non-LTE oracle against physics fixed independently of it:
tabulated hydrogen oscillator strengths, the Planck limits, a Saha special case,
Boltzmann ratios, detailed balance, the collision-dominated limit, the two-level
closed form, and E1 by quadrature."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

from oracle import nlte
from paper_2408_14425_b300 import workloads as W

ATOM = W.h3_atom()


def test_oscillator_strengths_match_hydrogen():
    """A_ul -> f_lu conversion (with g = 2n^2) against the tabulated hydrogen values
    Ly-alpha 0.4162, Ly-beta 0.07910, H-alpha 0.6407; the model's A and rounded level
    energies reproduce them to about one per cent."""
    f = [L["f_lu"] for L in nlte.line_constants(ATOM)]
    np.testing.assert_allclose(f, [0.4162, 0.07910, 0.6407], rtol=1.2e-2)
    lam_nm = [nlte.C / L["nu0"] * 1e9 for L in nlte.line_constants(ATOM)]
    np.testing.assert_allclose(lam_nm, [121.57, 102.57, 656.28], rtol=2e-3)


def test_planck_limits():
    T = 5000.0
    nu_lo = 1e9
    rj = 2 * nu_lo ** 2 * nlte.KB * T / nlte.C ** 2
    assert nlte.planck_nu(nu_lo, T) == pytest.approx(rj, rel=1e-4, abs=0)
    nu_hi = 3e15
    wien = 2 * nlte.H * nu_hi ** 3 / nlte.C ** 2 * math.exp(-nlte.H * nu_hi / (nlte.KB * T))
    assert nlte.planck_nu(nu_hi, T) == pytest.approx(wien, rel=1e-12, abs=0)


def test_saha_golden_ratio_point():
    """Where the Saha factor equals n_H, x^2/(1-x) = 1, so x = (sqrt 5 - 1)/2."""
    nH = 1e18

    def phi(T):
        return (2 * math.pi * nlte.ME * nlte.KB * T / nlte.H ** 2) ** 1.5 * \
            math.exp(-nlte.CHI_H / (nlte.KB * T))

    T = optimize.brentq(lambda t: math.log(phi(t) / nH), 3000.0, 3e5, xtol=1e-10)
    ne, n_atom = nlte.saha_hydrogen(np.array([T]), np.array([nH]))
    x = (math.sqrt(5) - 1) / 2
    assert ne[0] / nH == pytest.approx(x, rel=1e-9, abs=0)
    assert n_atom[0] / nH == pytest.approx(1 - x, rel=1e-9, abs=0)


def test_saha_hot_limit_keeps_digits():
    ne, n_atom = nlte.saha_hydrogen(np.array([1e6]), np.array([6e15]))
    phi = (2 * math.pi * nlte.ME * nlte.KB * 1e6 / nlte.H ** 2) ** 1.5 * \
        math.exp(-nlte.CHI_H / (nlte.KB * 1e6))
    # fully ionised: n_HI = n_e n_p / phi with n_e = n_p -> n_H
    assert n_atom[0] == pytest.approx(6e15 ** 2 / phi, rel=1e-6, abs=0)
    assert n_atom[0] > 0


def test_lte_boltzmann_ratios():
    T = np.array([6000.0, 2e4, 1e5])
    pops = nlte.lte_populations(ATOM, T, np.array([1.0, 2.0, 3.0]))
    np.testing.assert_allclose(pops.sum(axis=0), [1.0, 2.0, 3.0], rtol=1e-14)
    for lo, up in [(0, 1), (0, 2), (1, 2)]:
        dE = (ATOM["E_eV"][up] - ATOM["E_eV"][lo]) * nlte.EV
        expect = ATOM["g"][up] / ATOM["g"][lo] * np.exp(-dE / (nlte.KB * T))
        np.testing.assert_allclose(pops[up] / pops[lo], expect, rtol=1e-12)


def test_profile_normalisation():
    T = np.array([6000.0, 1e4, 3e4, 1e6])
    for (nu, w), phi in zip(nlte.frequency_grid(ATOM), nlte.profiles(ATOM, T)):
        np.testing.assert_allclose(np.sum(w[:, None] * phi, axis=0), 1.0, rtol=1e-13)
    # at T_ref the grid spans +-5 Doppler widths: the raw Gaussian already integrates to 1
    L = nlte.line_constants(ATOM)[0]
    nu, w = nlte.frequency_grid(ATOM)[0]
    dnu = L["nu0"] / nlte.C * math.sqrt(2 * nlte.KB * 1e4 / (ATOM["mass_amu"] * nlte.AMU))
    raw = np.exp(-((nu - L["nu0"]) / dnu) ** 2) / (math.sqrt(math.pi) * dnu)
    assert np.sum(w * raw) == pytest.approx(1.0, abs=1e-6)


def test_source_function_at_lte_is_planck():
    T = np.array([6000.0, 8000.0, 2e4])
    pops = nlte.lte_populations(ATOM, T, np.ones(3) * 1e17)
    for L, S in zip(nlte.line_constants(ATOM), nlte.line_source_function(ATOM, pops)):
        np.testing.assert_allclose(S, nlte.planck_nu(L["nu0"], T), rtol=1e-12)
    chi, eta = nlte.emis_opac(ATOM, T, pops)
    npl = ATOM["n_per_line"]
    for li, L in enumerate(nlte.line_constants(ATOM)):
        sl = slice(li * npl, (li + 1) * npl)
        np.testing.assert_allclose(eta[sl] / chi[sl],
                                   np.broadcast_to(nlte.planck_nu(L["nu0"], T), chi[sl].shape),
                                   rtol=1e-12)


def _planck_J(T):
    npl = ATOM["n_per_line"]
    return np.concatenate([np.repeat(nlte.planck_nu(L["nu0"], T)[None, :], npl, axis=0)
                           for L in nlte.line_constants(ATOM)], axis=0)


def test_detailed_balance_gives_lte_for_any_operator():
    """J = B_nu0(T) on every line wavelength and LTE previous populations: the MALI rates
    balance line by line for any Lambda*, so the solution is LTE."""
    rng = np.random.default_rng(1)
    T = rng.uniform(5000, 3e4, 50)
    nH = 10 ** rng.uniform(15, 18, 50)
    ne, n_atom = nlte.saha_hydrogen(T, nH)
    lte = nlte.lte_populations(ATOM, T, n_atom)
    J = _planck_J(T)
    alo = rng.uniform(0, 1, J.shape)
    new, dmax = nlte.stat_eq(ATOM, T, ne, n_atom, J, alo, lte)
    np.testing.assert_allclose(new, lte, rtol=1e-10)
    assert dmax < 1e-10


def test_collision_dominated_limit_is_lte():
    T = np.array([6000.0, 1e4, 5e4])
    n_atom = np.array([1e17, 1e16, 1e12])
    lte = nlte.lte_populations(ATOM, T, n_atom)
    start = lte * np.array([[1.0], [3.0], [0.1]])
    J = np.zeros((3 * ATOM["n_per_line"], 3))
    new, _ = nlte.stat_eq(ATOM, T, np.full(3, 1e32), n_atom, J, None, start)
    np.testing.assert_allclose(new, lte, rtol=1e-6)


def test_two_level_closed_form():
    atom2 = {"E_eV": [0.0, 10.2], "g": [2.0, 8.0], "lines": [(0, 1, 4.7e8)], "n_per_line": 21,
             "x_max": 5.0, "T_ref": 1e4, "mass_amu": 1.00794}
    T = np.array([7000.0, 1.5e4])
    ne = np.array([1e16, 3e17])
    n_atom = np.array([1e17, 5e16])
    Jval = np.array([3e-12, 8e-10])
    J = np.repeat(Jval[None, :], 21, axis=0)
    start = nlte.lte_populations(atom2, T, n_atom)
    new, _ = nlte.stat_eq(atom2, T, ne, n_atom, J, None, start)
    L = nlte.line_constants(atom2)[0]
    (Clu, Cul), = nlte.collision_rates(atom2, T, ne)
    ratio = (L["Blu"] * Jval + Clu) / (L["A"] + L["Bul"] * Jval + Cul)
    np.testing.assert_allclose(new[1] / new[0], ratio, rtol=1e-12)
    np.testing.assert_allclose(new.sum(axis=0), n_atom, rtol=1e-14)


def test_rate_matrix_columns_conserve():
    rng = np.random.default_rng(4)
    T = rng.uniform(6000, 1e5, 30)
    nH = 10 ** rng.uniform(15, 18, 30)
    ne, n_atom = nlte.saha_hydrogen(T, nH)
    pops = nlte.lte_populations(ATOM, T, n_atom)
    J = _planck_J(T) * rng.uniform(0.1, 2.0, (63, 30))
    G = nlte.rate_matrix(ATOM, T, ne, J, rng.uniform(0, 1, (63, 30)), pops)
    np.testing.assert_allclose(G.sum(axis=1), 0.0, atol=1e-9 * np.abs(G).max())
    off = G.copy()
    for i in range(3):
        off[:, i, i] = 0
    assert np.all(off >= 0)


def test_van_regemorter_gaunt_factor():
    """P(y) = max(0.2, 0.276 e^y E1(y)) with E1 by direct quadrature."""
    for y in [0.01, 0.1, 0.5, 1.0, 3.0, 20.0]:
        e1 = integrate.quad(lambda t: math.exp(-t) / t, y, math.inf, limit=200)[0]
        assert nlte.van_regemorter_P(y) == pytest.approx(max(0.2, 0.276 * math.exp(y) * e1),
                                                         rel=1e-8, abs=0)
    assert nlte.van_regemorter_P(50.0) == 0.2


def test_collision_rates_detailed_balance_and_scaling():
    T = np.array([8000.0, 2e5])
    ne = np.array([1e16, 2e16])
    for L, (Clu, Cul) in zip(nlte.line_constants(ATOM), nlte.collision_rates(ATOM, T, ne)):
        g = ATOM["g"]
        np.testing.assert_allclose(Clu / Cul, g[L["up"]] / g[L["lo"]] *
                                   np.exp(-L["dE"] / (nlte.KB * T)), rtol=1e-12)
    # proportional to n_e
    c1 = nlte.collision_rates(ATOM, T, ne)[0][1]
    c2 = nlte.collision_rates(ATOM, T, 3 * ne)[0][1]
    np.testing.assert_allclose(c2, 3 * c1, rtol=1e-14)
    # the thermal constant of the rate coefficient: h^2/((2 pi m_e)^1.5 k^0.5) = 8.629e-6 cgs
    assert nlte.BETA_COLL == pytest.approx(8.629e-12, rel=1e-3, abs=0)


def test_nlte_iteration_reaches_a_fixed_point():
    T, nH, vox = W.prominence_slab(n=32, half_width=6, blend=2, wander=2)
    pops, hist = nlte.nlte_iterate(ATOM, T, nH, vox, 4, max_iter=60, tol=1e-3)
    assert hist[-1] < 1e-3
    assert len(hist) < 60
    ne, n_atom = nlte.saha_hydrogen(T.ravel(), nH.ravel())
    np.testing.assert_allclose(pops.sum(axis=0), n_atom, rtol=1e-12)
    assert np.all(pops > 0)


# ---------------------------------------------------------------------------
# absolute scales: line opacity/emissivity and the collision rates
# ---------------------------------------------------------------------------

# classical oscillator cross-section per unit oscillator strength, SI:
# integral of sigma(nu) dnu = e^2 / (4 eps0 m_e c) f  (pi e^2 / (m_e c) f in cgs)
SIGMA_CLASSICAL = nlte.QE ** 2 / (4.0 * nlte.EPS0 * nlte.ME * nlte.C)    # m^2 Hz
F_TABLE = [0.4162, 0.07910, 0.6407]     # Ly-alpha, Ly-beta, H-alpha (hydrogen, tabulated)


def _random_state(n, seed):
    rng = np.random.default_rng(seed)
    T = rng.uniform(5000, 1e5, n)
    pops = 10 ** rng.uniform(10, 17, (3, n))          # arbitrary, not LTE
    return T, pops


def test_integrated_line_opacity_is_the_classical_oscillator_cross_section():
    """Sec. 3.2's chi at the line wavelengths, integrated over the line's frequency grid with
    its trapezoid weights, equals the classical oscillator cross-section times the
    stimulated-emission-corrected lower population:
        integral chi dnu = e^2 / (4 eps0 m_e c) f_lu (n_l - n_u g_l / g_u),
    with f_lu once from the oracle's own A -> f conversion (tight) and once from the tabulated
    hydrogen values (to the ~1 % that the model's rounded A and energies allow).  Dropping the
    h nu / 4 pi factor, mis-normalising phi, or a wrong B_lu (a missing c or nu power) fails it
    by orders of magnitude."""
    T, pops = _random_state(40, 7)
    chi, _ = nlte.emis_opac(ATOM, T, pops)
    npl = ATOM["n_per_line"]
    g = np.asarray(ATOM["g"])
    for li, (L, (nu, w)) in enumerate(zip(nlte.line_constants(ATOM), nlte.frequency_grid(ATOM))):
        integral = np.sum(w[:, None] * chi[li * npl:(li + 1) * npl], axis=0)
        corrected = pops[L["lo"]] - pops[L["up"]] * g[L["lo"]] / g[L["up"]]
        np.testing.assert_allclose(integral, SIGMA_CLASSICAL * L["f_lu"] * corrected, rtol=1e-12)
        np.testing.assert_allclose(integral, SIGMA_CLASSICAL * F_TABLE[li] * corrected,
                                   rtol=1.2e-2)


def test_lyman_alpha_line_centre_cross_section():
    """A printed textbook number: the Ly-alpha line-centre absorption cross-section of a
    thermal Gaussian profile is 5.9e-14 cm^2 (T / 1e4 K)^(-1/2).  chi per ground-state atom at
    the line-centre grid point (no upper population, T = T_ref so the grid spans +-5 Doppler
    widths and the renormalisation is ~1e-6) must give it; at 4e4 K it halves."""
    npl = ATOM["n_per_line"]
    centre = npl // 2
    for T, expect_cm2 in [(1e4, 5.9e-14), (4e4, 2.95e-14)]:
        pops = np.array([[1.0], [0.0], [0.0]])
        chi, _ = nlte.emis_opac(ATOM, np.array([T]), pops)
        sigma_cm2 = chi[centre, 0] * 1e4                 # m^2 -> cm^2 per atom
        assert sigma_cm2 == pytest.approx(expect_cm2, rel=1e-2, abs=0)


def test_emitted_power_is_spontaneous_decay_energy():
    """Energy conservation of spontaneous emission: 4 pi integral eta dnu = n_u A_ul h nu0 (every
    decay emits one photon of h nu0, isotropically).  A missing 1/(4 pi) or a profile that does
    not integrate to one fails it."""
    T, pops = _random_state(40, 8)
    _, eta = nlte.emis_opac(ATOM, T, pops)
    npl = ATOM["n_per_line"]
    for li, (L, (nu, w)) in enumerate(zip(nlte.line_constants(ATOM), nlte.frequency_grid(ATOM))):
        power = 4.0 * math.pi * np.sum(w[:, None] * eta[li * npl:(li + 1) * npl], axis=0)
        np.testing.assert_allclose(power, pops[L["up"]] * L["A"] * nlte.H * L["nu0"], rtol=1e-12)


def test_collision_rate_matches_van_regemorter_textbook_form():
    """Van Regemorter's downward rate in its usual cgs form,
        C_ul = 20.6 lambda^3 n_e T^(-1/2) A_ul P(y)   (lambda in cm, n_e in cm^-3, s^-1),
    which follows from the collision strength (8 pi / sqrt 3)(E_Ryd / dE) g_l f_lu P(y) with
    the thermal rate coefficient; the printed 20.6 carries three digits.  A wrong power of
    E_Ryd / dE (off by 1.13-7.2 on these lines), a dropped 8 pi / sqrt 3 or a wrong power of
    T fails it."""
    T = np.array([6000.0, 2e4, 1e5, 1e6])
    ne = np.array([1e16, 3e17, 1e15, 5e14])                        # m^-3
    for L, (Clu, Cul) in zip(nlte.line_constants(ATOM), nlte.collision_rates(ATOM, T, ne)):
        lam_cm = nlte.H * nlte.C / L["dE"] * 100.0
        y = L["dE"] / (nlte.KB * T)
        textbook = 20.6 * lam_cm ** 3 * (ne * 1e-6) / np.sqrt(T) * L["A"] * \
            nlte.van_regemorter_P(y)
        np.testing.assert_allclose(Cul, textbook, rtol=3e-3)


def _iterate(T, nH, vox, use_operator, tol, max_iter):
    from oracle import rc_solve
    n = T.shape[0]
    ne, n_atom = nlte.saha_hydrogen(T.ravel(), nH.ravel())
    pops = nlte.lte_populations(ATOM, T, n_atom)
    hist = []
    for _ in range(max_iter):
        chi, eta = nlte.emis_opac(ATOM, T, pops)
        J, alo, _ = rc_solve(chi.reshape(-1, n, n), eta.reshape(-1, n, n), 4, voxel=vox,
                             want_alo=True)
        pops, d = nlte.stat_eq(ATOM, T, ne, n_atom, J.reshape(chi.shape),
                               alo.reshape(chi.shape) if use_operator else None, pops)
        hist.append(d)
        if d < tol:
            break
    return pops, hist


def test_mali_and_lambda_iteration_share_the_fixed_point():
    """Sec. 3.3: the approximate operator only changes how fast the iteration moves, not where
    it ends -- at convergence J_eff + Lambda* S equals the formal solution's J, so MALI with
    Lambda* != 0 and plain Lambda iteration (Lambda* = 0) must reach the same populations.
    On a 16^2 slab at 1/100 of the prominence densities (line-core optical depth ~0.3 per
    voxel, thick across the sheet) both are run to a 1e-9 change: the populations agree to
    1e-6, and MALI needs a fraction of the iterations.  Swapping (1 - Lambda-bar) for
    Lambda-bar in the downward rate, or dropping the Lambda* S_dagger term of J_eff, moves one
    of the two fixed points and fails it."""
    T, nH, vox = W.prominence_slab(n=16, half_width=3.2, blend=2, wander=1, nH_cool=1e16,
                                   nH_lo=1e13, nH_hi=1e16)
    p_mali, h_mali = _iterate(T, nH, vox, True, 1e-9, 120)
    p_lam, h_lam = _iterate(T, nH, vox, False, 1e-9, 600)
    assert h_mali[-1] < 1e-9 and h_lam[-1] < 1e-9
    np.testing.assert_allclose(p_mali, p_lam, rtol=1e-6)
    assert len(h_mali) * 4 < len(h_lam)


def test_line_integrals_over_disjoint_ranges_add_up():
    """The rates see the radiation field only through each line's two integrals; with the
    profile normalised over the whole line, the integrals over disjoint wavelength ranges
    (the split between processes) add up to the line's, and the rate matrix built from them
    equals the one built from all wavelengths at once."""
    rng = np.random.default_rng(9)
    T = rng.uniform(6000, 3e4, 25)
    nH = 10 ** rng.uniform(15, 18, 25)
    ne, _ = nlte.saha_hydrogen(T, nH)
    J = _planck_J(T) * rng.uniform(0.2, 2.0, (63, 25))
    aloc = rng.uniform(0, 1, (63, 25))
    full = nlte.line_integrals(ATOM, T, J, aloc)
    parts = sum(nlte.line_integrals(ATOM, T, J[a:b], aloc[a:b], a)
                for a, b in [(0, 17), (17, 40), (40, 63)])
    np.testing.assert_allclose(parts, full, rtol=1e-14)
    np.testing.assert_allclose(nlte.rate_matrix_from_integrals(ATOM, T, ne, parts),
                               nlte.rate_matrix_eff(ATOM, T, ne, J, aloc), rtol=1e-13)
    # Lambda* = 0: the second integral is the profile's integral, 1
    np.testing.assert_allclose(nlte.line_integrals(ATOM, T, J, None)[:, 1], 1.0, rtol=1e-14)
