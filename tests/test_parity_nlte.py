"""Parity of the CUDA non-LTE pieces (through the C ABI) with the FP64 oracle.

FP64 kernels (LTE start, statistical equilibrium) must match the oracle to 1e-10;
FP32 outputs (chi, eta) to 1e-6; the MALI cascade-0 outputs (J_eff, 1 - Lambda*) to the
formal-solution tolerance 1e-3; populations after whole iterations (FP32 formal solution
inside) to the population tolerance 1e-4 relative.
"""
import numpy as np
import pytest

import oracle
from oracle import nlte
from paper_2408_14425_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ATOM = W.h3_atom()


def _rcx():
    from paper_2408_14425_b300 import build, rcx
    build.build()
    return rcx


def _slab(n=48, seed=11):
    return W.prominence_slab(n=n, seed=seed, half_width=n / 5, blend=3, wander=3)


def _dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def test_lte_start_matches_oracle():
    rcx = _rcx()
    atom = rcx.Atom(ATOM)
    T, nH, _ = _slab(64)
    ne, na, pops = atom.lte(_dev(T), _dev(nH))
    ne_r, na_r = nlte.saha_hydrogen(T.ravel(), nH.ravel())
    pops_r = nlte.lte_populations(ATOM, T, na_r)
    np.testing.assert_allclose(ne.cpu().numpy(), ne_r, rtol=1e-12)
    np.testing.assert_allclose(na.cpu().numpy(), na_r, rtol=1e-12)
    np.testing.assert_allclose(pops.cpu().numpy(), pops_r, rtol=1e-12)


@pytest.mark.parametrize("n_per_line", [21, 20, 7])
def test_emis_opac_matches_oracle(n_per_line):
    """Gaussian profiles on the line grids (odd and even point counts: the kernel walks the
    symmetric grid from its centre) and the emissivity/opacity against the FP64 oracle."""
    atom_d = dict(ATOM, n_per_line=n_per_line)
    rcx = _rcx()
    atom = rcx.Atom(atom_d)
    T, nH, _ = _slab(64)
    ne_r, na_r = nlte.saha_hydrogen(T.ravel(), nH.ravel())
    rng = np.random.default_rng(2)
    pops = nlte.lte_populations(atom_d, T, na_r) * rng.uniform(0.5, 2.0, (3, T.size))
    chi, eta = atom.emis_opac(_dev(T), _dev(pops))
    chi_r, eta_r = nlte.emis_opac(atom_d, T, pops)
    np.testing.assert_allclose(chi.cpu().numpy(), chi_r.astype(np.float32), rtol=2e-6)
    np.testing.assert_allclose(eta.cpu().numpy(), eta_r.astype(np.float32), rtol=2e-6)


def test_stat_eq_matches_oracle_on_the_same_inputs():
    """Same FP32 (J_eff, 1 - Lambda*) into both: the rates and the FP64 solve agree."""
    rcx = _rcx()
    atom = rcx.Atom(ATOM)
    T, nH, vox = _slab(40)
    ne_r, na_r = nlte.saha_hydrogen(T.ravel(), nH.ravel())
    pops0 = nlte.lte_populations(ATOM, T, na_r)
    chi_r, eta_r = nlte.emis_opac(ATOM, T, pops0)
    J_r, alo_r, _ = oracle.rc_solve(chi_r.reshape(-1, *T.shape), eta_r.reshape(-1, *T.shape), 5,
                                    voxel=vox, want_alo=True)
    Jeff, aloc = nlte.effective_inputs(ATOM, J_r.reshape(chi_r.shape), alo_r.reshape(chi_r.shape),
                                       pops0)
    Jeff32 = Jeff.astype(np.float32)
    aloc32 = aloc.astype(np.float32)
    new_r, dmax_r = nlte.stat_eq_eff(ATOM, T, ne_r, na_r, Jeff32.astype(np.float64),
                                     aloc32.astype(np.float64), pops0)
    pops = _dev(pops0)
    dmax = atom.stat_eq(_dev(T), _dev(ne_r), _dev(na_r), _dev(Jeff32, torch.float32),
                        _dev(aloc32, torch.float32), pops)
    np.testing.assert_allclose(pops.cpu().numpy(), new_r, rtol=1e-10)
    assert dmax == pytest.approx(dmax_r, rel=1e-8, abs=0)
    # plain Lambda iteration (no operator): J as J_eff, alo_c = NULL
    new_l, _ = nlte.stat_eq(ATOM, T, ne_r, na_r, J_r.reshape(chi_r.shape).astype(np.float32)
                            .astype(np.float64), None, pops0)
    pops = _dev(pops0)
    atom.stat_eq(_dev(T), _dev(ne_r), _dev(na_r),
                 _dev(J_r.reshape(chi_r.shape), torch.float32), None, pops)
    np.testing.assert_allclose(pops.cpu().numpy(), new_l, rtol=1e-10)


def test_mali_outputs_match_oracle():
    """J_eff = J - Lambda* S_local and 1 - Lambda* from the cascade-0 kernel."""
    rcx = _rcx()
    T, nH, vox = _slab(48)
    ne_r, na_r = nlte.saha_hydrogen(T.ravel(), nH.ravel())
    pops0 = nlte.lte_populations(ATOM, T, na_r)
    chi_r, eta_r = nlte.emis_opac(ATOM, T, pops0)
    chi32 = chi_r.astype(np.float32).reshape(-1, *T.shape)
    eta32 = eta_r.astype(np.float32).reshape(-1, *T.shape)
    J_r, alo_r, _ = oracle.rc_solve(chi32.astype(np.float64), eta32.astype(np.float64), 5,
                                    voxel=vox, want_alo=True)
    S_loc = np.where(chi32 > 0, eta32.astype(np.float64) / chi32.astype(np.float64), 0.0)
    Jeff_r = J_r - alo_r * S_loc
    plan = rcx.Plan(T.shape[1], T.shape[0], 5, voxel_size=vox)
    J, Jeff, aloc = plan.formal_solve_mali(_dev(chi32, torch.float32), _dev(eta32, torch.float32))
    J, Jeff, aloc = J.cpu().numpy(), Jeff.cpu().numpy(), aloc.cpu().numpy()
    for name, a, b in [("J", J, J_r), ("J_eff", Jeff, Jeff_r), ("1-alo", aloc, 1.0 - alo_r)]:
        floor = 1e-7 * np.abs(b).max(axis=(1, 2), keepdims=True)
        bad = np.abs(a - b) > 1e-3 * np.abs(b) + floor
        assert not bad.any(), f"{name}: {bad.sum()} cells off, max rel " \
                              f"{(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)).max():.2e}"


@pytest.mark.parametrize("n_iter", [1, 6])
def test_whole_iterations_match_oracle(n_iter):
    """n_iter iterations of the whole loop (emissivity, FP32 formal solution, FP64 update)
    from LTE on a 32^2 slab: populations within 1e-4 of the FP64 oracle's iterates."""
    rcx = _rcx()
    T, nH, vox = _slab(32)
    atom = rcx.Atom(ATOM)
    ne, na, pops = atom.lte(_dev(T), _dev(nH))
    plan = rcx.Plan(32, 32, 4, voxel_size=vox)
    conv, it, hist = rcx.nlte_solve(plan, atom, _dev(T), ne, na, pops, tol=1e-30,
                                    max_iter=n_iter)
    assert not conv and it == n_iter
    pops_r, hist_r = nlte.nlte_iterate(ATOM, T, nH, vox, 4, max_iter=n_iter, tol=1e-30)
    g = pops.cpu().numpy()
    rel = np.abs(g - pops_r) / np.abs(pops_r)
    assert rel.max() < 1e-4, f"max rel population difference {rel.max():.3e}"
    np.testing.assert_allclose(hist, hist_r, rtol=1e-2)


def test_nlte_converges_on_a_slab():
    rcx = _rcx()
    T, nH, vox = _slab(64)
    atom = rcx.Atom(ATOM)
    ne, na, pops = atom.lte(_dev(T), _dev(nH))
    plan = rcx.Plan(64, 64, 5, voxel_size=vox)
    conv, it, hist = rcx.nlte_solve(plan, atom, _dev(T), ne, na, pops, tol=1e-3, max_iter=200)
    assert conv and hist[-1] < 1e-3
    p = pops.cpu().numpy()
    np.testing.assert_allclose(p.sum(axis=0), na.cpu().numpy(), rtol=1e-12)
    assert np.all(p > 0)


def test_resume_from_checkpoint_equals_straight_run(tmp_path):
    """Populations are the whole state of the iteration: 3 iterations, a checkpoint written
    and read back, 2 more iterations give bit for bit the populations of 5 straight ones."""
    from paper_2408_14425_b300 import checkpoint
    rcx = _rcx()
    T, nH, vox = _slab(48)
    atom = rcx.Atom(ATOM)
    plan = rcx.Plan(48, 48, 5, voxel_size=vox)
    Td = _dev(T)
    ne, na, straight = atom.lte(Td, _dev(nH))
    rcx.nlte_solve(plan, atom, Td, ne, na, straight, tol=1e-30, max_iter=5)
    _, _, pops = atom.lte(Td, _dev(nH))
    _, it, hist = rcx.nlte_solve(plan, atom, Td, ne, na, pops, tol=1e-30, max_iter=3)
    f = str(tmp_path / "nlte.npz")
    checkpoint.save(f, pops, it, hist)
    resumed, it0, _ = checkpoint.load(f, device="cuda")
    assert it0 == 3
    rcx.nlte_solve(plan, atom, Td, ne, na, resumed, tol=1e-30, max_iter=2)
    np.testing.assert_array_equal(resumed.cpu().numpy(), straight.cpu().numpy())


def test_full_size_slab_converges_with_sampled_oracle_updates():
    """The non-LTE slab at its full size (512^2, 63 wavelengths, 6 cascades, the bench's
    seed 11) converges to max relative change < 1e-3; populations stay positive and sum to
    n_atom in every cell; and for 64 sampled cells the statistical-equilibrium update from
    the converged state, fed the GPU's FP32 (J_eff, 1 - Lambda*), equals the FP64 oracle's
    update of those cells to 1e-10."""
    rcx = _rcx()
    T, nH, vox = W.prominence_slab(n=512, seed=11)
    atom = rcx.Atom(ATOM)
    Td = _dev(T)
    ne, na, pops = atom.lte(Td, _dev(nH))
    plan = rcx.Plan(512, 512, 6, voxel_size=vox)
    conv, it, hist = rcx.nlte_solve(plan, atom, Td, ne, na, pops, tol=1e-3, max_iter=300)
    assert conv and hist[-1] < 1e-3
    P = pops.cpu().numpy()
    na_h = na.cpu().numpy()
    assert np.all(P > 0)
    np.testing.assert_allclose(P.sum(axis=0), na_h, rtol=1e-12)
    chi, eta = atom.emis_opac(Td, pops)
    nl = chi.shape[0]
    _, J_eff, alo_c = plan.formal_solve_mali(chi.reshape(nl, 512, 512), eta.reshape(nl, 512, 512))
    J_eff = J_eff.reshape(nl, -1)
    alo_c = alo_c.reshape(nl, -1)
    new = pops.clone()
    atom.stat_eq(Td, ne, na, J_eff, alo_c, new)
    cells = np.random.default_rng(4).choice(512 * 512, 64, replace=False)
    new_r, _ = nlte.stat_eq_eff(ATOM, T.ravel()[cells], ne.cpu().numpy()[cells], na_h[cells],
                                J_eff.cpu().numpy()[:, cells].astype(np.float64),
                                alo_c.cpu().numpy()[:, cells].astype(np.float64), P[:, cells])
    np.testing.assert_allclose(new.cpu().numpy()[:, cells], new_r, rtol=1e-10)


def test_c3_crop_populations_over_a_converged_length_run():
    """The non-LTE workload's slab (seed 11, 5.7 km voxels, 63 wavelengths, 6 cascades)
    cropped to its central 128^2 (the cool sheet, its transition region and corona): 24
    whole iterations from LTE -- as many as the full slab needs to reach a 1e-3 change --
    on the GPU and in the FP64 oracle.  The populations must agree element by element
    within the population tolerance 1e-4 relative, and the GPU's history of maximum changes
    must follow the oracle's."""
    rcx = _rcx()
    T5, nH5, vox = W.prominence_slab(n=512, seed=11)
    crop = (slice(192, 320), slice(192, 320))
    T = np.ascontiguousarray(T5[crop])
    nH = np.ascontiguousarray(nH5[crop])
    atom = rcx.Atom(ATOM)
    ne, na, pops = atom.lte(_dev(T), _dev(nH))
    plan = rcx.Plan(128, 128, 6, voxel_size=vox)
    conv, it, hist = rcx.nlte_solve(plan, atom, _dev(T), ne, na, pops, tol=1e-30, max_iter=24)
    assert it == 24
    pops_r, hist_r = nlte.nlte_iterate(ATOM, T, nH, vox, 6, max_iter=24, tol=1e-30)
    g = pops.cpu().numpy()
    rel = np.abs(g - pops_r) / np.abs(pops_r)
    assert rel.max() < 1e-4, f"max rel population difference {rel.max():.3e}"
    np.testing.assert_allclose(hist, hist_r, rtol=2e-2)


def test_c3_full_size_J_in_si_units():
    """The formal solution of the full 512^2 slab in SI units (chi in m^-1, 5.7 km voxels,
    intensities per unit frequency ~1e-9..1e-13), at the LTE populations: for the Ly-alpha
    core, a Ly-alpha wing point and the H-alpha core, J from the GPU (all 63 wavelengths in
    one solve) equals the FP64 oracle's cell by cell within the FP32 tolerance 1e-3."""
    rcx = _rcx()
    T, nH, vox = W.prominence_slab(n=512, seed=11)
    atom = rcx.Atom(ATOM)
    Td = _dev(T)
    ne, na, pops = atom.lte(Td, _dev(nH))
    chi, eta = atom.emis_opac(Td, pops)
    nl = chi.shape[0]
    chi = chi.reshape(nl, 512, 512)
    eta = eta.reshape(nl, 512, 512)
    plan = rcx.Plan(512, 512, 6, voxel_size=vox)
    J = plan.formal_solve(chi, eta).cpu().numpy()
    chi_h = chi.cpu().numpy()
    eta_h = eta.cpu().numpy()
    for lam in (10, 2, 52):
        J_r, _, _ = oracle.rc_solve(chi_h[lam:lam + 1].astype(np.float64),
                                    eta_h[lam:lam + 1].astype(np.float64), 6, voxel=vox)
        ref = J_r[0]
        floor = 1e-7 * np.abs(ref).max()
        bad = np.abs(J[lam] - ref) > 1e-3 * np.abs(ref) + floor
        assert not bad.any(), f"lambda {lam}: {bad.sum()} cells off, max rel " \
                              f"{(np.abs(J[lam] - ref) / np.abs(ref)).max():.2e}"


def test_line_integrals_split_equals_stat_eq():
    """rc_line_integrals over disjoint wavelength ranges, summed (the all-reduce of a
    wavelength split), then rc_stat_eq_integrals: the populations of rc_stat_eq to 1e-12;
    with one range over all wavelengths, bit for bit.  The integrals match the FP64
    oracle's on the same FP32 inputs to 1e-10, the bar of the other FP64 kernels here (the
    kernel's Gaussian profile comes from a ratio recurrence a few ulps from the direct
    exponentials)."""
    rcx = _rcx()
    atom = rcx.Atom(ATOM)
    T, nH, vox = _slab(48)
    Td = _dev(T)
    ne, na, pops0 = atom.lte(Td, _dev(nH))
    chi, eta = atom.emis_opac(Td, pops0)
    nl = chi.shape[0]
    plan = rcx.Plan(48, 48, 5, voxel_size=vox)
    _, J_eff, alo_c = plan.formal_solve_mali(chi.reshape(nl, 48, 48), eta.reshape(nl, 48, 48))
    J_eff, alo_c = J_eff.reshape(nl, -1), alo_c.reshape(nl, -1)
    ref = pops0.clone()
    d_ref = atom.stat_eq(Td, ne, na, J_eff, alo_c, ref)
    whole = atom.line_integrals(Td, J_eff, alo_c, 0)
    one = pops0.clone()
    d_one = atom.stat_eq_integrals(Td, ne, na, whole, one)
    assert torch.equal(one, ref) and d_one == d_ref
    split = atom.line_integrals(Td, J_eff[:30].contiguous(), alo_c[:30].contiguous(), 0) + \
        atom.line_integrals(Td, J_eff[30:].contiguous(), alo_c[30:].contiguous(), 30)
    two = pops0.clone()
    atom.stat_eq_integrals(Td, ne, na, split, two)
    np.testing.assert_allclose(two.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12)
    w_r = nlte.line_integrals(ATOM, T, J_eff.cpu().numpy().astype(np.float64),
                              alo_c.cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(whole.cpu().numpy(), w_r, rtol=1e-10)


def test_sharded_driver_in_one_process_equals_nlte_solve():
    """The wavelength-split driver with a single process (one range, no collective) walks
    the same iteration as rc_nlte_solve: same iteration count and populations."""
    from paper_2408_14425_b300 import distributed
    rcx = _rcx()
    atom = rcx.Atom(ATOM)
    T, nH, vox = _slab(48)
    Td = _dev(T)
    plan = rcx.Plan(48, 48, 5, voxel_size=vox)
    ne, na, pops = atom.lte(Td, _dev(nH))
    conv, it, hist = rcx.nlte_solve(plan, atom, Td, ne, na, pops, tol=1e-3, max_iter=100)
    _, _, pops2 = atom.lte(Td, _dev(nH))
    ops = distributed.GpuOps(plan, atom, Td, ne, na)
    conv2, it2, hist2 = distributed.nlte_solve_sharded(ops, atom.n_lambda, pops2, tol=1e-3,
                                                       max_iter=100)
    assert conv and conv2 and it == it2
    np.testing.assert_allclose(pops2.cpu().numpy(), pops.cpu().numpy(), rtol=1e-13)
