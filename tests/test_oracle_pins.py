"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses an independent
construction (fine-step integration of the RTE, closed forms of the disc
problems, algebraic identities of the interval representation, a recursive
construction of the cascade merge, brute-force long characteristics).
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_2408_14425_b300 import workloads as W


def _random_field(n, seed, chi_lo=1e-3, chi_hi=3.0, s_lo=0.1, s_hi=10.0):
    rng = np.random.default_rng(seed)
    chi = 10 ** rng.uniform(np.log10(chi_lo), np.log10(chi_hi), size=(n, n))
    S = 10 ** rng.uniform(np.log10(s_lo), np.log10(s_hi), size=(n, n))
    return chi, S * chi


def _fine_integral(chi, eta, o, w, a, b, h=4e-6, chunk=2_000_000):
    """Independent RTE integral along o + t w, t in [a, b]: midpoint sampling of the
    voxel field on a very fine uniform sub-grid (no face-crossing logic at all).
    Each face crossed adds an error below h times the jump of the integrand."""
    nz, nx = chi.shape
    if not np.isfinite(b):
        corners = np.array([[0, 0], [nx, 0], [0, nz], [nx, nz]], dtype=np.float64)
        b = a + np.max(np.hypot(corners[:, 0] - o[0], corners[:, 1] - o[1])) + 1.0
    n_sub = int(np.ceil((b - a) / h))
    h = (b - a) / n_sub
    I = 0.0
    tau_acc = 0.0
    for s0 in range(0, n_sub, chunk):
        t = a + h * (np.arange(s0, min(n_sub, s0 + chunk)) + 0.5)
        x = o[0] + t * w[0]
        z = o[1] + t * w[1]
        inside = (x >= 0) & (x < nx) & (z >= 0) & (z < nz)
        ix = np.clip(np.floor(x).astype(np.int64), 0, nx - 1)
        iz = np.clip(np.floor(z).astype(np.int64), 0, nz - 1)
        c = np.where(inside, chi[iz, ix], 0.0)
        e = np.where(inside, eta[iz, ix], 0.0)
        dtau = c * h
        cs = np.cumsum(dtau)
        tau_before = tau_acc + np.concatenate([[0.0], cs[:-1]])
        with np.errstate(divide="ignore", invalid="ignore"):
            contrib = np.where(c > 0, e / np.where(c > 0, c, 1) * -np.expm1(-dtau), e * h)
        I += float(np.sum(np.exp(-tau_before) * contrib))
        tau_acc += float(cs[-1])
    return I, tau_acc


# ---------------------------------------------------------------------------
# cascade geometry (Sec. 2.3, Eq. 12-14)
# ---------------------------------------------------------------------------

def test_intervals_contiguous_and_scaling():
    C = 8
    for rule in (0, 1):
        prev_b = None
        for i in range(C):
            a, b = oracle.interval(i, C, 1.0, 4, rule)
            if i == 0:
                assert a == 0.0  # t_0 = 0 (Eq. 13)
            else:
                assert a == prev_b  # shells [t_i, t_{i+1}] tile the line
            if i == C - 1:
                assert math.isinf(b)  # top cascade leaves the domain (Sec. 2.3)
            elif rule == 0:
                assert b - a == pytest.approx(4.0 ** i)  # t_i ~ 2^(alpha i), alpha = 2
            else:
                assert b == pytest.approx(4.0 ** i)
            prev_b = b
    # branching 2 (alpha = 1): lengths double
    a2, b2 = oracle.interval(3, 6, 1.5, 2, 0)
    assert b2 - a2 == pytest.approx(1.5 * 8)


def test_ray_counts_equal_per_cascade_alpha2():
    """With alpha = 2 in 2D every cascade holds N_C0 rays (Sec. 2.4)."""
    n = 256
    n0 = n * n * 4
    for i in range(8):
        P = oracle.probes(n, i)
        assert P * P * oracle.dirs(4, 4, i) == n0
    # alpha = 1: N_Ci halves per cascade and the sum stays below 2 N_C0 (Eq. 14)
    tot = sum(oracle.probes(n, i) ** 2 * oracle.dirs(4, 2, i) for i in range(8))
    assert oracle.probes(n, 1) ** 2 * oracle.dirs(4, 2, 1) == n0 // 2
    assert tot < 2 * n0


def test_children_tile_parent_cone():
    for i, W in enumerate([4, 16, 64]):
        for k in range(W):
            lo, hi = 2 * math.pi * k / W, 2 * math.pi * (k + 1) / W
            th_parent = math.atan2(*oracle.direction(k, W)[::-1]) % (2 * math.pi)
            assert lo < th_parent < hi
            kids = [math.atan2(*oracle.direction(4 * k + c, 4 * W)[::-1]) % (2 * math.pi)
                    for c in range(4)]
            assert all(lo < t < hi for t in kids)
            # equally spaced, each covers a quarter of the parent cone
            d = np.diff(sorted(kids))
            assert np.allclose(d, (hi - lo) / 4)


# ---------------------------------------------------------------------------
# one radiance interval (Eq. 9, Eq. 16)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_march_matches_fine_rte_integration(seed):
    chi, eta = _random_field(16, seed, chi_hi=0.5)
    rng = np.random.default_rng(100 + seed)
    th = rng.uniform(0, 2 * np.pi)
    w = (math.cos(th), math.sin(th))
    o = rng.uniform(-2, 18, size=2)
    a = rng.uniform(0, 4)
    b = math.inf if seed % 3 == 0 else a + rng.uniform(2, 20)
    I, tau, n = oracle.march(chi, eta, o, w, a, b)
    I_ref, tau_ref = _fine_integral(chi, eta, o, w, a, b)
    assert n > 0 or I == 0.0
    assert tau == pytest.approx(tau_ref, rel=1e-5, abs=1e-12)
    assert I == pytest.approx(I_ref, rel=1e-5, abs=1e-12)


def test_march_crossing_count_is_cells_visited():
    chi = np.ones((32, 32))
    # a ray across the whole grid from x=0: cells = 1 + x faces + z faces
    o = (0.0, 3.3)
    th = 0.3
    w = (math.cos(th), math.sin(th))
    _, _, n = oracle.march(chi, chi, o, w, 0.0, math.inf)
    t_exit = min(32 / w[0], (32 - 3.3) / w[1])
    x_end = o[0] + t_exit * w[0]
    z_end = o[1] + t_exit * w[1]
    expect = 1 + (math.ceil(x_end) - 1) + (math.ceil(z_end) - 1 - 3)
    assert n == expect


def test_uniform_medium_closed_form():
    chi = np.full((20, 20), 0.37)
    eta = np.full((20, 20), 0.37 * 4.0)
    for th in (0.1, 1.0, 2.5, 4.0):
        w = (math.cos(th), math.sin(th))
        I, tau, _ = oracle.march(chi, eta, (10.0, 10.0), w, 1.0, 6.5)
        assert tau == pytest.approx(0.37 * 5.5, rel=1e-13, abs=0)
        assert I == pytest.approx(4.0 * -math.expm1(-0.37 * 5.5), rel=1e-13, abs=0)


def test_zero_opacity_cells_emit_eta_ds():
    chi = np.zeros((8, 8))
    eta = np.full((8, 8), 0.25)
    I, tau, _ = oracle.march(chi, eta, (4.0, 4.0), (1.0, 0.0), 0.0, 2.5)
    assert tau == 0.0
    assert I == pytest.approx(0.25 * 2.5, rel=1e-14, abs=0)


def test_free_space_outside_domain():
    chi, eta = _random_field(8, 3)
    I, tau, n = oracle.march(chi, eta, (4.0, 4.0), (0.6, 0.8), 20.0, math.inf)
    assert (I, tau, n) == (0.0, 0.0, 0)


@pytest.mark.parametrize("seed", range(5))
def test_merge_splitting_invariance(seed):
    """M(R_{a,b}, R_{b,c}) = R_{a,c} (Eq. 11); fixes which interval attenuates which."""
    chi, eta = _random_field(24, seed)
    rng = np.random.default_rng(seed)
    th = rng.uniform(0, 2 * np.pi)
    w = (math.cos(th), math.sin(th))
    o = rng.uniform(6, 18, size=2)
    a, b, c = 0.3, 0.3 + rng.uniform(1, 5), 12.0
    near = oracle.march(chi, eta, o, w, a, b)[:2]
    far = oracle.march(chi, eta, o, w, b, c)[:2]
    whole = oracle.march(chi, eta, o, w, a, c)[:2]
    Im, tm = oracle.merge(near, far)
    assert tm == pytest.approx(whole[1], rel=1e-12, abs=0)
    assert Im == pytest.approx(whole[0], rel=1e-12, abs=0)
    # the order printed in Eq. 11 (far attenuated by nothing, near by far) is not
    # the radiation arriving at the probe for an inhomogeneous medium
    swapped = far[0] + math.exp(-far[1]) * near[0]
    assert abs(swapped - whole[0]) > 1e-6 * abs(whole[0])


@pytest.mark.parametrize("x", [0.5, 2.0, 7.25])
def test_shift_identity(x):
    """R_{a+x,b+x}(p, w) = R_{a,b}(p + x w, w) (Eq. 10)."""
    chi, eta = _random_field(24, 11)
    th = 0.77
    w = (math.cos(th), math.sin(th))
    p = np.array([5.3, 4.1])
    r1 = oracle.march(chi, eta, p, w, 1.0 + x, 9.0 + x)
    r2 = oracle.march(chi, eta, p + x * np.array(w), w, 1.0, 9.0)
    assert r1[0] == pytest.approx(r2[0], rel=1e-12, abs=0)
    assert r1[1] == pytest.approx(r2[1], rel=1e-12, abs=0)


# ---------------------------------------------------------------------------
# the whole cascade (Sec. 2.3.1, 2.5, Eq. 1)
# ---------------------------------------------------------------------------

def _tree_rc(chi, eta, C, W0=4, B=4, L0=1.0, fix=False):
    """The cascade merge built recursively from probe *positions* (Sec. 2.3.1):
    a cascade-i ray merges with the child-cone average of the four cascade-(i+1)
    probes that bracket its probe, bilinearly weighted, clamped at the edges.
    With fix, the ray is traced from its start to the start of each upper probe's
    child interval and merged there (the bilinear fix of Sec. 2.5)."""
    nz, nx = chi.shape
    memo = {}

    def upper_probes(x, n, i):
        """Bracketing cascade-(i+1) probe indices and weights along one axis."""
        s = 2 ** (i + 1)
        P = -(-n // s)
        pos = [(j + 0.5) * s for j in range(P)]
        if x <= pos[0]:
            return [(0, 1.0)]
        if x >= pos[-1]:
            return [(P - 1, 1.0)]
        j = max(j for j in range(P) if pos[j] <= x)
        f = (x - pos[j]) / s
        return [(j, 1.0 - f), (j + 1, f)]

    def V(i, px, pz, k):
        key = (i, px, pz, k)
        if key in memo:
            return memo[key]
        s = 2 ** i
        x, z = (px + 0.5) * s, (pz + 0.5) * s
        Wi = W0 * B ** i
        th = 2 * math.pi * (k + 0.5) / Wi
        a, b = oracle.interval(i, C, L0, B, 0)
        w = (math.cos(th), math.sin(th))
        if fix and i < C - 1:
            a_up = oracle.interval(i + 1, C, L0, B, 0)[0]
            su = 2 ** (i + 1)
            A = np.array([x + a * w[0], z + a * w[1]])
            total = 0.0
            for jx, wx in upper_probes(x, nx, i):
                for jz, wz in upper_probes(z, nz, i):
                    Bp = np.array([(jx + 0.5) * su + a_up * w[0], (jz + 0.5) * su + a_up * w[1]])
                    L = float(np.hypot(*(Bp - A)))
                    Ib, tb, _ = oracle.march(chi, eta, A, (Bp - A) / L, 0.0, L)
                    avg = sum(V(i + 1, jx, jz, B * k + c) for c in range(B)) / B
                    total += wx * wz * (Ib + math.exp(-tb) * avg)
            memo[key] = total
            return total
        I, tau, _ = oracle.march(chi, eta, (x, z), w, a, b)
        if i < C - 1:
            up = 0.0
            for jx, wx in upper_probes(x, nx, i):
                for jz, wz in upper_probes(z, nz, i):
                    up += wx * wz * sum(V(i + 1, jx, jz, B * k + c) for c in range(B)) / B
            I = I + math.exp(-tau) * up
        memo[key] = I
        return I

    J = np.zeros_like(chi)
    for iz in range(nz):
        for ix in range(nx):
            J[iz, ix] = sum(V(0, ix, iz, k) for k in range(W0)) / W0
    return J


@pytest.mark.parametrize("n,C,fix", [(16, 4, False), (12, 3, False), (16, 4, True),
                                     (12, 3, True)])
def test_rc_matches_recursive_construction(n, C, fix):
    chi, eta = _random_field(n, 5 + n, chi_hi=1.0)
    J, _, _ = oracle.rc_solve(chi, eta, C, bilinear_fix=fix)
    J_tree = _tree_rc(chi, eta, C, fix=fix)
    np.testing.assert_allclose(J, J_tree, rtol=1e-12, atol=0)


def test_bilinear_fix_removes_ringing():
    """Sec. 2.5: the bilinear fix suppresses the ringing of the basic method around an
    opaque disc; the pixelisation bias (above the theory curve) stays."""
    n, R = 128, 10.0
    chi, eta = W.opaque_disc_field(n, R, chi_disc=100.0)
    c = n / 2
    stats = {}
    for fix in (False, True):
        J, _, _ = oracle.rc_solve(chi, eta, 6, bilinear_fix=fix)
        rel = []
        for ix in range(int(c + R + 3), n - 12):
            d = ix + 0.5 - c
            Jrc = 0.5 * (J[int(c), ix] + J[int(c) - 1, ix])
            rel.append(Jrc / (math.asin(R / math.hypot(d, 0.5)) / math.pi) - 1)
        stats[fix] = np.array(rel)
    assert stats[True].std() < 0.5 * stats[False].std()
    assert stats[True].max() < stats[False].max()
    assert stats[True].min() > 0.0


def test_thick_limit_J_equals_local_source():
    """Deep optical thickness: J -> S of the cell itself (PAPER: J of Eq. 1 with Eq. 16)."""
    rng = np.random.default_rng(3)
    chi = np.full((32, 32), 80.0)
    S = rng.uniform(0.1, 10, size=(32, 32))
    J, _, _ = oracle.rc_solve(chi, S * chi, 5)
    np.testing.assert_allclose(J, S, rtol=1e-12)


def test_alo_is_local_coefficient_of_J():
    """With a single cascade extending to infinity, a lone emitting cell c gives
    J_c = S_c Lambda*_c exactly, with Lambda* = 1 - exp(-chi d) (reading of Eq. 17)."""
    rng = np.random.default_rng(9)
    chi = 10 ** rng.uniform(-2, 0.5, size=(10, 10))
    eta = np.zeros_like(chi)
    c = (4, 6)
    eta[c] = 3.0 * chi[c]
    J, alo, _ = oracle.rc_solve(chi, eta, 1, want_alo=True)
    assert J[c] == pytest.approx(3.0 * alo[c], rel=1e-13, abs=0)
    d = 0.5 * math.sqrt(2.0)  # centre to edge along the cascade-0 diagonals
    assert alo[c] == pytest.approx(-math.expm1(-chi[c] * d), rel=1e-13, abs=0)


def test_thin_disc_closed_form():
    """Optically thin uniform disc: J(d) = eta (2R/pi) E(d/R) inside and
    (2 eta/pi) int_0^asin(R/d) sqrt(R^2 - d^2 sin^2 phi) dphi outside."""
    n, R = 64, 12.0
    chi, eta = W.thin_disc_field(n, R)
    J, _, _ = oracle.rc_solve(chi, eta, 5)
    c = n / 2
    errs_in, errs_out = [], []
    for ix in range(int(c), n - 4):
        d = ix + 0.5 - c
        Jrc = 0.5 * (J[int(c), ix] + J[int(c) - 1, ix])  # average the two rows straddling z = c
        if d < R - 1.5:
            ref = (2 * R / math.pi) * special.ellipe((d / R) ** 2)
            errs_in.append(Jrc / ref - 1)
        elif d > R + 1.5:
            phim = math.asin(R / d)
            ref = (2 / math.pi) * integrate.quad(
                lambda p: math.sqrt(max(R * R - d * d * math.sin(p) ** 2, 0.0)), 0, phim)[0]
            errs_out.append(Jrc / ref - 1)
    assert max(abs(e) for e in errs_in) < 0.02
    assert max(abs(e) for e in errs_out) < 0.10
    assert np.median(np.abs(errs_out)) < 0.04


def test_opaque_disc_falloff_band():
    """Sec. 2.5 circle test: outside an opaque S = 1 disc in vacuum J = asin(R/d)/pi.
    The basic RC result lies above theory (pixelised disc) with ringing of up to
    about ten per cent."""
    n, R = 128, 10.0
    chi, eta = W.opaque_disc_field(n, R, chi_disc=100.0)
    J, _, _ = oracle.rc_solve(chi, eta, 6)
    c = n / 2
    rel = []
    for ix in range(int(c + R + 3), n - 12):
        d = ix + 0.5 - c
        Jrc = 0.5 * (J[int(c), ix] + J[int(c) - 1, ix])
        d_true = math.hypot(d, 0.5)
        rel.append(Jrc / (math.asin(R / d_true) / math.pi) - 1)
    rel = np.array(rel)
    assert np.all(rel > -0.05)
    assert np.all(rel < 0.20)
    assert np.median(rel) > 0.0  # sits above the theory curve


def test_rc_close_to_long_characteristics():
    """RC against brute-force long characteristics (2048 angles) on a rough GRF field.
    The difference is the method's own approximation (interpolation, parallax):
    a few per cent typically (Sec. 2.5), larger at isolated dim cells."""
    n = 64
    chi, eta = W.grf_fields(n, 1, dtype=np.float64)
    chi = chi[0] * 1e-1
    eta = eta[0] * 1e-1
    J_rc, _, _ = oracle.rc_solve(chi, eta, 5)
    J_lc = oracle.lc_solve(chi, eta, 2048)
    rel = np.abs(J_rc / J_lc - 1)
    assert np.median(rel) < 0.03
    assert np.linalg.norm(J_rc - J_lc) / np.linalg.norm(J_lc) < 0.06


@pytest.mark.parametrize("n", [1, 2, 4, 8])
def test_gauss_radau_inclination_rule(n):
    """Fixed node at mu = 0, weights summing to 1, exact for polynomials up to degree 2n - 2
    on [0, 1] (Sec. 3.1 uses eight Gauss-Radau inclinations)."""
    mu, w = oracle.gauss_radau_inclinations(n)
    assert mu[0] == 0.0 and np.all(np.diff(mu) > 0) and mu[-1] < 1.0
    assert w.sum() == pytest.approx(1.0, rel=1e-12, abs=0)
    for p in range(2 * n - 1):
        assert np.sum(w * mu ** p) == pytest.approx(1.0 / (p + 1), rel=1e-11, abs=1e-14)
    if n > 1:   # and not beyond: degree 2n - 1 is not integrated exactly
        assert abs(np.sum(w * mu ** (2 * n - 1)) - 1.0 / (2 * n)) > 1e-12


def test_inclinations_thick_and_thin_limits():
    """Thick: J = S whatever the inclination.  Thin: every inclination adds the emission along
    a path 1/sqrt(1 - mu^2) longer, so J = J_flat * sum_j w_j / sqrt(1 - mu_j^2)."""
    rng = np.random.default_rng(8)
    S = rng.uniform(0.5, 2.0, (16, 16))
    chi = np.full((16, 16), 60.0)
    J, _ = oracle.rc_solve_inclined(chi, S * chi, 4, 8)
    np.testing.assert_allclose(J, S, rtol=1e-12)
    chi_t = np.full((16, 16), 1e-10)
    eta_t = rng.uniform(0.5, 2.0, (16, 16)) * 1e-10
    J_flat, _, _ = oracle.rc_solve(chi_t, eta_t, 4)
    J_inc, _ = oracle.rc_solve_inclined(chi_t, eta_t, 4, 8)
    mu, w = oracle.gauss_radau_inclinations(8)
    np.testing.assert_allclose(J_inc, J_flat * np.sum(w / np.sqrt(1 - mu ** 2)), rtol=1e-7)


def test_sparse_equals_dense_on_the_masked_field():
    """Sec. 3.5: with inactive cells transparent and only flagged probes computed, every
    active cell's J equals the dense solution of the masked field (flagged parents carry
    every dependency), inactive cells get 0, and the work falls with the active fraction."""
    rng = np.random.default_rng(12)
    n = 64
    chi, eta = _random_field(n, 21, chi_hi=1.0)
    T = 10 ** rng.uniform(3.5, 6.5, (n, n))
    x = np.arange(n) + 0.5
    active = (np.abs(x[None, :] - 20) < 6) | (np.hypot(x[None, :] - 45, x[:, None] - 40) < 7)
    J_s, rays = oracle.rc_solve_sparse(chi, eta, active, 5)
    J_d, _, _ = oracle.rc_solve(np.where(active, chi, 0.0), np.where(active, eta, 0.0), 5)
    assert np.all(np.isfinite(J_s))
    np.testing.assert_allclose(J_s[active], J_d[active], rtol=1e-14)
    assert np.all(J_s[~active] == 0.0)
    dense_rays = np.array([oracle.probes(n, i) ** 2 * oracle.dirs(4, 4, i) for i in range(5)])
    assert rays[0] == active.sum() * 4
    assert np.all(rays <= dense_rays) and rays.sum() < 0.8 * dense_rays.sum()
    del T


def test_emergent_front_to_back_equals_back_to_front():
    """Sec. 3.9: the single-pass front-to-back intensity equals the back-to-front march of
    the same ray, and the contribution function sums to it."""
    chi, eta = _random_field(24, 31)
    rng = np.random.default_rng(31)
    rays = []
    for _ in range(12):
        th = rng.uniform(0, 2 * np.pi)
        rays.append((rng.uniform(-3, 27), rng.uniform(-3, 27), math.cos(th), math.sin(th)))
    I, C = oracle.emergent(chi, eta, rays, want_contrib=True)
    for (ox, oz, wx, wz), Ii in zip(rays, I):
        assert Ii == pytest.approx(oracle.march(chi, eta, (ox, oz), (wx, wz), 0.0, math.inf)[0],
                                   rel=1e-12, abs=1e-300)
    assert C.sum() == pytest.approx(I.sum(), rel=1e-12, abs=0)


def test_emergent_uniform_slab_closed_form():
    """Through a uniform slab of depth D at inclination mu: I = S (1 - exp(-chi D / sqrt(1 - mu^2)))."""
    chi = np.full((8, 40), 0.3)
    eta = 0.3 * 2.0 * np.ones_like(chi)
    rays = [(x + 0.5, -1.0, 0.0, 1.0) for x in range(40)]
    for mu in (0.0, 0.6):
        I = oracle.emergent(chi, eta, rays, mu=mu)
        np.testing.assert_allclose(I, 2.0 * -np.expm1(-0.3 * 8 / math.sqrt(1 - mu * mu)), rtol=1e-12)
