"""Parity of the CUDA formal solution (through the C ABI) with the FP64 oracle.

Tolerance: J within 1e-3 relative in FP32 storage mode and 5e-3 with 16-bit
interval storage, element by element, with an absolute floor of 1e-7 of the
slab's largest J (cells darker than that carry no relative information in
FP32 after ~1e3 accumulated crossings).
"""
import numpy as np
import pytest

import oracle
from paper_2408_14425_b300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rcx():
    from paper_2408_14425_b300 import build, rcx
    build.build()
    return rcx


def _assert_close(J, J_ref, rtol, what=""):
    J = np.asarray(J, dtype=np.float64)
    J_ref = np.asarray(J_ref, dtype=np.float64)
    assert J.shape == J_ref.shape
    assert np.all(np.isfinite(J))
    floor = 1e-7 * np.max(np.abs(J_ref), axis=(-2, -1), keepdims=True)
    err = np.abs(J - J_ref)
    bad = err > rtol * np.abs(J_ref) + floor
    if bad.any():
        idx = np.argwhere(bad)[0]
        rel = (err / np.maximum(np.abs(J_ref), 1e-300)).max()
        raise AssertionError(f"{what}: {bad.sum()} cells out of tolerance, first at {tuple(idx)}: "
                             f"{J[tuple(idx)]} vs {J_ref[tuple(idx)]} (max rel {rel:.3e})")


def _solve(chi, eta, C, want_alo=False, **plan_kw):
    rcx = _rcx()
    nl, nz, nx = chi.shape
    p = rcx.Plan(nx, nz, C, **plan_kw)
    dchi = torch.from_numpy(np.ascontiguousarray(chi, dtype=np.float32)).cuda()
    deta = torch.from_numpy(np.ascontiguousarray(eta, dtype=np.float32)).cuda()
    out = p.formal_solve(dchi, deta, want_alo=want_alo)
    torch.cuda.synchronize()
    if want_alo:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy()


def _oracle(chi, eta, C, want_alo=False, **kw):
    # the oracle sees the same FP32 inputs, widened to FP64
    J, alo, _ = oracle.rc_solve(chi.astype(np.float64), eta.astype(np.float64), C,
                                want_alo=want_alo, **kw)
    return (J, alo) if want_alo else J


def test_disc_64_five_cascades():
    """64x64 disc, 1 wavelength, 5 cascades, W0 = 4, branching 4, interval 1 voxel."""
    chi, eta = W.disc_field()
    J, alo = _solve(chi, eta, 5, want_alo=True)
    J_ref, alo_ref = _oracle(chi, eta, 5, want_alo=True)
    _assert_close(J, J_ref, 1e-3, "J disc")
    _assert_close(alo, alo_ref, 1e-5, "alo disc")


@pytest.mark.parametrize("nx,nz,nl,C", [(96, 80, 7, 5), (130, 67, 5, 6), (33, 200, 3, 6)])
def test_grf_ragged_shapes(nx, nz, nl, C):
    """Non-square, non-power-of-two grids and a ragged last wavelength block."""
    chi, eta = W.grf_fields(nx, nl, nz=nz)
    J = _solve(chi, eta, C)
    _assert_close(J, _oracle(chi, eta, C), 1e-3, f"J grf {nx}x{nz}")


def test_grf_256_seven_cascades():
    chi, eta = W.grf_fields(256, 6)
    J, alo = _solve(chi, eta, 7, want_alo=True)
    J_ref, alo_ref = _oracle(chi, eta, 7, want_alo=True)
    _assert_close(J, J_ref, 1e-3, "J grf 256")
    _assert_close(alo, alo_ref, 1e-5, "alo grf 256")


@pytest.mark.parametrize("lb,vl", [(1, 1), (2, 2), (4, 1), (4, 4), (8, 4), (8, 8), (16, 2),
                                   (16, 4), (16, 8), (32, 1), (32, 4), (32, 8)])
def test_lane_layouts_agree(lb, vl):
    """Every lane layout (wavelengths per ray, per lane) computes each (ray, wavelength)
    with the same arithmetic, so the results are identical."""
    chi, eta = W.grf_fields(72, 9)
    J_ref = _solve(chi, eta, 5, lambda_block=8, lambda_per_lane=2)
    J = _solve(chi, eta, 5, lambda_block=lb, lambda_per_lane=vl)
    np.testing.assert_array_equal(J, J_ref)


def test_interval_rule_alternative():
    chi, eta = W.grf_fields(64, 2)
    J = _solve(chi, eta, 5, interval_rule=1)
    _assert_close(J, _oracle(chi, eta, 5, rule=1), 1e-3, "rule 1")


@pytest.mark.parametrize("C,W0,L0,voxel", [(1, 4, 1.0, 1.0), (2, 8, 1.5, 1.0), (4, 4, 2.0, 0.25),
                                           (6, 4, 1.0, 5.7e3)])
def test_plan_parameters(C, W0, L0, voxel):
    chi, eta = W.grf_fields(48, 2)
    if voxel != 1.0:
        chi = (chi / voxel).astype(np.float32)
        eta = (eta / voxel).astype(np.float32)
    J = _solve(chi, eta, C, dirs0=W0, interval0=L0, voxel_size=voxel)
    J_ref = _oracle(chi, eta, C, dirs0=W0, interval0=L0, voxel=voxel)
    _assert_close(J, J_ref, 1e-3, f"C={C} W0={W0} L0={L0} voxel={voxel}")


@pytest.mark.parametrize("nx,nz", [(1, 1), (1, 17), (23, 1), (2, 2)])
def test_degenerate_grids(nx, nz):
    rng = np.random.default_rng(nx * 100 + nz)
    chi = (10 ** rng.uniform(-3, 1, size=(2, nz, nx))).astype(np.float32)
    eta = (chi * rng.uniform(0.1, 10, size=chi.shape)).astype(np.float32)
    J = _solve(chi, eta, 4)
    _assert_close(J, _oracle(chi, eta, 4), 1e-3, f"{nx}x{nz}")


def test_zero_opacity_and_vacuum():
    """chi = 0 cells keep their emission (eta ds); an empty domain gives J = 0."""
    chi, eta = W.grf_fields(40, 2)
    chi[0, 10:20, 5:30] = 0.0
    J = _solve(chi, eta, 5)
    _assert_close(J, _oracle(chi, eta, 5), 1e-3, "chi=0 patch")
    z = np.zeros((1, 16, 16), np.float32)
    assert np.all(_solve(z, z, 3) == 0.0)


def test_zero_wavelengths_is_a_no_op():
    rcx = _rcx()
    p = rcx.Plan(16, 16, 3)
    e = torch.empty((0, 16, 16), dtype=torch.float32, device="cuda")
    J = p.formal_solve(e, e)
    assert J.shape == (0, 16, 16)


@pytest.mark.parametrize("prec,tol", [("f16", 5e-3), ("bf16", 5e-3)])
def test_reduced_precision_storage(prec, tol):
    chi, eta = W.grf_fields(128, 5)
    J = _solve(chi, eta, 6, precision=prec)
    _assert_close(J, _oracle(chi, eta, 6), tol, prec)


@pytest.mark.parametrize("nl", [37, 64, 100])
def test_host_buffer_entry_matches_device_entry(nl):
    """The host-buffer entry (chunks of 16 wavelengths at the ends, 32 between) gives the
    device entry's results bit for bit: 37 -> 16+16+5, 64 -> 16+32+16, 100 -> 16+32+32+16+4."""
    rcx = _rcx()
    chi, eta = W.grf_fields(64, nl)
    p = rcx.Plan(64, 64, 5)
    J_host, alo_host = p.formal_solve_host(chi, eta, want_alo=True)
    J_dev, alo_dev = p.formal_solve(torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda(),
                                    want_alo=True)
    np.testing.assert_array_equal(J_host, J_dev.cpu().numpy())
    np.testing.assert_array_equal(alo_host, alo_dev.cpu().numpy())


def test_full_size_1024_sampled_wavelengths():
    """The benchmark workload (1024^2, 64 wavelengths, 8 cascades) solved in one call;
    two of its wavelengths compared with the oracle cell by cell."""
    chi, eta = W.grf_fields(1024, 64)
    J = _solve(chi, eta, 8)
    for lam in (0, 45):
        J_ref = _oracle(chi[lam:lam + 1], eta[lam:lam + 1], 8)
        _assert_close(J[lam:lam + 1], J_ref, 1e-3, f"1024^2 lambda {lam}")


@pytest.mark.parametrize("nx,nz,nl,C", [(96, 80, 5, 5), (64, 64, 3, 5)])
def test_bilinear_fix_matches_oracle(nx, nz, nl, C):
    """Sec. 2.5's bilinear fix (four traced segments per ray below the top cascade)."""
    chi, eta = W.grf_fields(nx, nl, nz=nz)
    J = _solve(chi, eta, C, bilinear_fix=True)
    _assert_close(J, _oracle(chi, eta, C, bilinear_fix=True), 1e-3, f"fix {nx}x{nz}")


def test_bilinear_fix_circle_test():
    chi, eta = W.opaque_disc_field(128, 10.0, chi_disc=100.0)
    chi = chi[None].astype(np.float32)
    eta = eta[None].astype(np.float32)
    J = _solve(chi, eta, 6, bilinear_fix=True)
    _assert_close(J, _oracle(chi, eta, 6, bilinear_fix=True), 1e-3, "fix circle")


def test_bilinear_fix_rejects_the_operator_outputs():
    rcx = _rcx()
    p = rcx.Plan(16, 16, 3, bilinear_fix=True)
    x = torch.ones((1, 16, 16), device="cuda")
    with pytest.raises(rcx.RcError):
        p.formal_solve(x, x, want_alo=True)
    with pytest.raises(rcx.RcError):
        p.formal_solve_mali(x, x)


@pytest.mark.parametrize("n_incl,C,strips", [(8, 5, 0), (3, 4, 0), (3, 5, 3)])
def test_inclinations_match_oracle(n_incl, C, strips):
    """2D invariance (Sec. 3.1): Gauss-Radau inclinations, J and the diagonal operator (also
    with the cascades strip-split)."""
    chi, eta = W.grf_fields(80, 6, nz=72)
    J, alo = _solve(chi, eta, C, want_alo=True, n_incl=n_incl, strips=strips)
    J_ref, alo_ref = oracle.rc_solve_inclined(chi.astype(np.float64), eta.astype(np.float64), C,
                                              n_incl, want_alo=True)
    _assert_close(J, J_ref, 1e-3, f"J n_incl={n_incl}")
    _assert_close(alo, alo_ref, 1e-5, f"alo n_incl={n_incl}")


def test_inclinations_host_entry_and_mali():
    rcx = _rcx()
    chi, eta = W.grf_fields(48, 5)
    p = rcx.Plan(48, 48, 5, n_incl=4)
    J_host = p.formal_solve_host(chi, eta)
    dchi, deta = torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda()
    np.testing.assert_array_equal(J_host, p.formal_solve(dchi, deta).cpu().numpy())
    J, J_eff, alo_c = p.formal_solve_mali(dchi, deta)
    J_ref, alo_ref = oracle.rc_solve_inclined(chi.astype(np.float64), eta.astype(np.float64), 5, 4,
                                              want_alo=True)
    _assert_close(J.cpu().numpy(), J_ref, 1e-3, "mali J")
    _assert_close(alo_c.cpu().numpy(), 1.0 - alo_ref, 1e-3, "mali 1-alo")


def _mask(nx, nz, seed=0):
    x = np.arange(nx) + 0.5
    z = np.arange(nz) + 0.5
    X, Z = np.meshgrid(x, z)
    m = (np.abs(X - 0.3 * nx) < 0.08 * nx + 1) | (np.hypot(X - 0.7 * nx, Z - 0.6 * nz) < 0.12 * nx)
    return m


@pytest.mark.parametrize("nx,nz,C", [(64, 64, 5), (96, 70, 6)])
def test_sparse_matches_oracle(nx, nz, C):
    """Sec. 3.5: flagged probes only; active cells match the oracle, inactive cells are 0, and
    the flagged-probe counts equal the oracle's interval counts per direction."""
    rcx = _rcx()
    chi, eta = W.grf_fields(nx, 3, nz=nz)
    m = _mask(nx, nz)
    p = rcx.Plan(nx, nz, C)
    p.set_active(torch.from_numpy(m.astype(np.uint8)).cuda())
    J = p.formal_solve(torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda()).cpu().numpy()
    counts = p.active_probes()
    for lam in range(3):
        J_ref, rays = oracle.rc_solve_sparse(chi[lam].astype(np.float64), eta[lam].astype(np.float64),
                                             m, C)
        _assert_close(J[lam][None], J_ref[None], 1e-3, f"sparse lambda {lam}")
        assert np.all(J[lam][~m] == 0.0)
    dirs = [oracle.dirs(4, 4, i) for i in range(C)]
    assert counts[0] == m.sum()
    assert [int(r) // w for r, w in zip(rays, dirs)] == counts


@pytest.mark.parametrize("nx,nz,C,nl", [(96, 70, 6, 20), (160, 128, 7, 16)])
def test_sparse_march_equals_dense_march_on_the_masked_field(nx, nz, C, nl):
    """A sparse plan packs inactive cells as chi' = S = 0 and marches only the flagged probes.
    A dense plan marching the field with chi = eta = 0 outside the active set packs those
    cells at the opacity floor with S = 0, where a step changes nothing (e^{-dtau} rounds to
    1).  J on the active cells is bit-identical between the two, as are J_eff and
    1 - Lambda*: the flagged probes carry every interval the active cells merge."""
    rcx = _rcx()
    chi, eta = W.grf_fields(nx, nl, nz=nz)
    m = _mask(nx, nz)
    chi0, eta0 = chi * m[None], eta * m[None]
    sp = rcx.Plan(nx, nz, C)
    sp.set_active(torch.from_numpy(m.astype(np.uint8)).cuda())
    dn = rcx.Plan(nx, nz, C)
    out_s = sp.formal_solve_mali(torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda())
    out_d = dn.formal_solve_mali(torch.from_numpy(chi0).cuda(), torch.from_numpy(eta0).cuda())
    mm = torch.from_numpy(m).cuda()
    for a, b in zip(out_s, out_d):
        a, b = a[:, mm].cpu(), b[:, mm].cpu()
        assert torch.equal(a, b), f"max abs diff {(a - b).abs().max().item():.3e}"
    sp.close()
    dn.close()


def test_sparse_cleared_is_dense_again():
    rcx = _rcx()
    chi, eta = W.grf_fields(48, 2)
    dchi, deta = torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda()
    p = rcx.Plan(48, 48, 5)
    J0 = p.formal_solve(dchi, deta).cpu().numpy()
    p.set_active(torch.from_numpy(_mask(48, 48).astype(np.uint8)).cuda())
    p.formal_solve(dchi, deta)
    p.set_active(None)
    np.testing.assert_array_equal(p.formal_solve(dchi, deta).cpu().numpy(), J0)


def test_sparse_nlte_keeps_inactive_populations():
    rcx = _rcx()
    T, nH, vox = W.prominence_slab(n=48, half_width=10, blend=3, wander=3)
    atom = rcx.Atom(W.h3_atom())
    dT, dnH = torch.from_numpy(T).cuda(), torch.from_numpy(nH).cuda()
    ne, na, pops = atom.lte(dT, dnH)
    lte = pops.clone()
    plan = rcx.Plan(48, 48, 5, voxel_size=vox)
    active = torch.from_numpy((T < 2.5e5).astype(np.uint8)).cuda()
    plan.set_active(active)
    conv, it, hist = rcx.nlte_solve(plan, atom, dT, ne, na, pops, tol=1e-3, max_iter=200)
    assert conv
    inactive = active.cpu().numpy().ravel() == 0
    assert inactive.any()
    np.testing.assert_array_equal(pops.cpu().numpy()[:, inactive], lte.cpu().numpy()[:, inactive])


@pytest.mark.parametrize("mu", [0.0, 0.5])
def test_emergent_intensity_and_contribution_function(mu):
    """Sec. 3.9: front-to-back long characteristics along given rays, with the contribution
    function summed per cell."""
    rcx = _rcx()
    chi, eta = W.grf_fields(64, 5, nz=48)
    rng = np.random.default_rng(5)
    th = 0.3
    rays = [(x + 0.5, -0.5, np.sin(th), np.cos(th)) for x in range(-10, 64)]
    for _ in range(40):
        a = rng.uniform(0, 2 * np.pi)
        rays.append((rng.uniform(-4, 68), rng.uniform(-4, 52), np.cos(a), np.sin(a)))
    rays = np.array(rays, dtype=np.float32)
    p = rcx.Plan(64, 48, 3)
    I, C = p.emergent(torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda(),
                      torch.from_numpy(rays).cuda(), mu=mu, want_contrib=True)
    I, C = I.cpu().numpy(), C.cpu().numpy()
    for lam in range(5):
        I_ref, C_ref = oracle.emergent(chi[lam].astype(np.float64), eta[lam].astype(np.float64),
                                       rays.astype(np.float64), mu=mu, want_contrib=True)
        _assert_close(I[lam][None, None], I_ref[None, None], 1e-3, f"I lambda {lam}")
        _assert_close(C[lam][None], C_ref[None], 2e-3, f"contribution lambda {lam}")
        assert C[lam].sum() == pytest.approx(I[lam].sum(), rel=1e-4, abs=0)


@pytest.mark.parametrize("mu", [0.0, 0.5])
def test_emergent_intensity_in_pieces(mu):
    """Without the contribution function each ray's span in the box is marched as 4 pieces by
    neighbouring lane groups and composed front to back (Eq. 11).  I matches the oracle and
    the single-pass march (the contribution-function call) to FP32 rounding, for rays that
    start outside or inside the domain, run along an axis, graze a corner or miss it, with 17
    wavelengths (a ragged second block)."""
    rcx = _rcx()
    nl = 17
    chi, eta = W.grf_fields(64, nl, nz=48)
    rng = np.random.default_rng(9)
    rays = [(x + 0.5, -0.5, 0.0, 1.0) for x in range(0, 64, 7)]          # along z
    rays += [(-0.5, z + 0.25, 1.0, 0.0) for z in range(0, 48, 5)]        # along x
    rays += [(-1.0, -1.0, 0.6, 0.8), (70.0, 60.0, -0.8, -0.6), (-5.0, 50.0, 1.0, 0.0),
             (64.0, 0.0, 0.7071068, -0.7071068)]                         # corner, miss
    for _ in range(60):
        a = rng.uniform(0, 2 * np.pi)
        rays.append((rng.uniform(-4, 68), rng.uniform(-4, 52), np.cos(a), np.sin(a)))
    rays = np.array(rays, dtype=np.float32)
    p = rcx.Plan(64, 48, 3)
    dchi, deta, drays = (torch.from_numpy(x).cuda() for x in (chi, eta, rays))
    I = p.emergent(dchi, deta, drays, mu=mu, want_contrib=False).cpu().numpy()
    I1, _ = p.emergent(dchi, deta, drays, mu=mu, want_contrib=True)
    I1 = I1.cpu().numpy()
    _assert_close(I[None], I1[None], 1e-4, "pieces vs single pass")
    for lam in (0, 8, 16):
        I_ref = oracle.emergent(chi[lam].astype(np.float64), eta[lam].astype(np.float64),
                                rays.astype(np.float64), mu=mu, want_contrib=False)
        _assert_close(I[lam][None, None], I_ref[None, None], 1e-3, f"I lambda {lam}")


@pytest.mark.parametrize("n,C,launched", [(64, 5, 4), (64, 7, 4), (1024, 8, 7), (100, 4, 4)])
def test_free_space_cascades_are_not_launched(n, C, launched):
    """Sec. 3.4: an interval beyond the farthest box corner from every probe of its cascade
    lies in free space, so top cascades whose intervals all do are identically zero and are
    not launched; the results still match the oracle, which marches them.
    64^2: cascade 4 starts at 85 > 79.2 (probe (8, 8) to corner (64, 64)), cascades 5-6
    further out; cascade 3 starts at 21 < 84.9.  1024^2: cascade 7 starts at 5461 > 1357.6,
    cascade 6 at 1365 < 1402.9.  100^2: cascade 3 starts at 21 < 135.8."""
    rcx = _rcx()
    p = rcx.Plan(n, n, C, strips=1)                   # one launch per live cascade
    chi, eta = W.grf_fields(n, 1 if n > 100 else 2)
    dchi, deta = torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda()
    J = p.formal_solve(dchi, deta)
    torch.cuda.synchronize()
    assert p.last_launch_count() == 1 + launched      # pack + live cascades
    if n <= 100:
        _assert_close(J.cpu().numpy(), _oracle(chi, eta, C), 1e-3, f"{n} C{C}")


@pytest.mark.parametrize("nx,nz,C,strips,prec,nl", [(96, 80, 5, 3, "f32", 5), (130, 67, 6, 4, "f32", 5),
                                                    (64, 64, 5, 16, "f32", 5), (96, 80, 5, 2, "bf16", 5),
                                                    (96, 80, 5, 3, "f32", 40)])
def test_strip_split_march_matches_unsplit_and_oracle(nx, nz, C, strips, prec, nl):
    """Every cascade >= 1 marched strip by strip (one launch per vertical strip, partial
    (I, T) composed front to back or back to front by the ray's x direction) gives the
    unsplit result up to FP32 rounding, and the oracle's.  With 40 wavelengths one strip
    launch covers three wavelength blocks, the last one ragged."""
    rcx = _rcx()
    chi, eta = W.grf_fields(nx, nl, nz=nz)
    dchi, deta = torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda()
    whole = rcx.Plan(nx, nz, C, precision=prec, strips=1)
    split = rcx.Plan(nx, nz, C, precision=prec, strips=strips)
    J1, A1 = whole.formal_solve(dchi, deta, want_alo=True)
    J2, A2 = split.formal_solve(dchi, deta, want_alo=True)
    torch.cuda.synchronize()
    J1, J2 = J1.cpu().numpy(), J2.cpu().numpy()
    # the strip faces are entered at t computed from the face itself and left at t from the
    # DDA's face count: the two differ by an ulp of t, so one piece per face moves by it
    _assert_close(J2, J1, 1e-4 if prec == "f32" else 2e-3, "split vs whole")
    np.testing.assert_array_equal(A2.cpu().numpy(), A1.cpu().numpy())   # cascade 0 is not split
    _assert_close(J2, _oracle(chi, eta, C), 1e-3 if prec == "f32" else 5e-3, "split vs oracle")


def test_strip_split_with_sparsity_and_mali():
    rcx = _rcx()
    chi, eta = W.grf_fields(96, 4, nz=72)
    dchi, deta = torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda()
    active = np.zeros((72, 96), dtype=np.uint8)
    active[10:50, 20:70] = 1
    out = []
    for strips in (1, 3):
        p = rcx.Plan(96, 72, 5, strips=strips)
        p.set_active(torch.from_numpy(active).cuda())
        out.append([t.cpu().numpy() for t in p.formal_solve_mali(dchi, deta)])
    for a, b in zip(*out):
        _assert_close(b, a, 1e-4, "sparse split vs whole")


def test_strip_split_automatic_at_1024():
    """At 1024^2 with 16 wavelengths per block (128 MiB of packed field) cascade 5 (intervals
    from 341 to the far corner) runs in 2 strips; cascade 4 (256 voxels long) and cascade 6
    (38 voxels inside the domain) do not.  Each strip launch covers all three wavelength
    blocks (their partial (I, T), 3 x 512 MiB, fits the 8 GiB it keeps for them)."""
    rcx = _rcx()
    chi, eta = W.grf_fields(1024, 48, lambdas=range(48))
    dchi, deta = torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda()
    auto = rcx.Plan(1024, 1024, 8)
    whole = rcx.Plan(1024, 1024, 8, strips=1)
    Ja = auto.formal_solve(dchi, deta)
    n_auto = auto.last_launch_count()
    Jw = whole.formal_solve(dchi, deta)
    n_whole = whole.last_launch_count()
    torch.cuda.synchronize()
    assert n_whole == 1 + 7 and n_auto == n_whole + 1     # pack + cascades 6..0; c5 in 2 strips
    assert auto.scratch_bytes() - whole.scratch_bytes() == 3 * 4194304 * 16 * 8
    _assert_close(Ja.cpu().numpy(), Jw.cpu().numpy(), 5e-4, "auto strips vs whole")


def test_large_thick_uniform_domain():
    """4096^2, 16 wavelengths, 9 cascades (a 2 GiB field block, so the long cascades run in
    16 strips; cascade 8 lies in free space): in a uniform medium of optical depth 1 per
    voxel, J equals S wherever every ray has crossed 40 voxels before leaving the domain
    (exp(-40) below FP32 resolution)."""
    rcx = _rcx()
    n, nl = 4096, 16
    S = np.linspace(0.5, 2.0, nl, dtype=np.float32)
    chi = torch.ones((nl, n, n), device="cuda")
    eta = chi * torch.from_numpy(S).cuda()[:, None, None]
    p = rcx.Plan(n, n, 9)
    J = p.formal_solve(chi, eta)
    torch.cuda.synchronize()
    inner = J[:, 40:-40, 40:-40]
    rel = (inner / torch.from_numpy(S).cuda()[:, None, None] - 1.0).abs().max().item()
    assert rel < 1e-5, rel
    assert p.last_launch_count() > 1 + 8     # strips on the long cascades
    del chi, eta, J


@pytest.mark.parametrize("nx,nz,C,strips,prec,nl", [
    (96, 80, 5, 0, "f32", 20), (130, 67, 6, 4, "f32", 17), (64, 64, 5, 3, "bf16", 16),
    (257, 129, 7, 0, "f16", 33), (200, 200, 6, 2, "f32", 1)])
def test_shared_dda_march_equals_lane_group_march(nx, nz, C, strips, prec, nl):
    """The shared-DDA march (one warp walks 32 rays' DDA into shared memory and replays it
    for their wavelengths) performs the same arithmetic as the lane-group march: J, the
    operator outputs and the merged result agree bit for bit, unsplit and strip by strip,
    on ragged grids whose ray counts leave partial warps and CTAs."""
    rcx = _rcx()
    rng = np.random.default_rng(nx + nz)
    chi = (10 ** rng.uniform(-4, 1.5, (nl, nz, nx))).astype(np.float32)
    eta = (chi * 10 ** rng.uniform(-1, 1, chi.shape)).astype(np.float32)
    dchi, deta = torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda()
    out = []
    for mode in (rcx.Plan.MARCH_LANE_GROUP, rcx.Plan.MARCH_SHARED_DDA,
                 rcx.Plan.MARCH_SHARED_DDA_ALL):
        p = rcx.Plan(nx, nz, C, precision=prec, strips=strips)
        p.set_march(mode)
        assert p.march() == mode
        J, Jeff, aloc = p.formal_solve_mali(dchi, deta)
        out.append((J.cpu(), Jeff.cpu(), aloc.cpu()))
        p.close()
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert torch.equal(a, b), f"max abs diff {(a - b).abs().max().item():.3e}"


def test_pipelined_host_solves_equal_blocking_ones():
    """rc_formal_solve_host_async: three consecutive calls on different inputs (each cut into
    16 + 32 + 16-wavelength chunks whose staging buffers alternate across the calls) give,
    after rc_plan_wait, the J and Lambda* of one blocking rc_formal_solve_host per input, bit
    for bit."""
    rcx = _rcx()
    n, nl = 96, 64
    ins = []
    for seed in range(3):
        rng = np.random.default_rng(50 + seed)
        chi = (10 ** rng.uniform(-4, 1.5, (nl, n, n))).astype(np.float32)
        ins.append((chi, (chi * 10 ** rng.uniform(-1, 1, chi.shape)).astype(np.float32)))
    plan = rcx.Plan(n, n, 6)
    outs = [(np.full((nl, n, n), np.nan, np.float32), np.full((nl, n, n), np.nan, np.float32))
            for _ in ins]
    for (chi, eta), (J, alo) in zip(ins, outs):
        plan.formal_solve_host_async(chi, eta, J, alo)
    plan.wait()
    for (chi, eta), (J, alo) in zip(ins, outs):
        J_ref, alo_ref = plan.formal_solve_host(chi, eta, want_alo=True)
        np.testing.assert_array_equal(J, J_ref)
        np.testing.assert_array_equal(alo, alo_ref)


def test_march_modes_agree_at_full_size():
    """The headline grid (1024^2, 8 cascades, cascade 5 strip-split automatically) with 32
    wavelengths (two 16-wavelength blocks): the lane-group march, the default (shared DDA on
    the short cascades) and the shared DDA everywhere (its strip kernels included) give the
    same J bit for bit."""
    rcx = _rcx()
    from paper_2408_14425_b300 import workloads
    chi, eta = workloads.grf_fields(1024, 32)
    dchi, deta = torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda()
    out = []
    for mode in (rcx.Plan.MARCH_LANE_GROUP, rcx.Plan.MARCH_SHARED_DDA,
                 rcx.Plan.MARCH_SHARED_DDA_ALL):
        p = rcx.Plan(1024, 1024, 8)
        p.set_march(mode)
        out.append(p.formal_solve(dchi, deta).cpu())
        p.close()
    assert torch.equal(out[0], out[1]) and torch.equal(out[0], out[2])


@pytest.mark.parametrize("nx,nz,C,prec,nl", [
    (1024, 1024, 8, "f32", 16), (1100, 900, 8, "bf16", 16), (300, 260, 6, "f16", 33),
    (280, 280, 6, "f32", 5)])
def test_top_cascade_over_listed_ctas_equals_every_cta(nx, nz, C, prec, nl):
    """The highest launched cascade marches only the CTAs with a ray that can reach the box
    (the others store R = 0 through a cleared buffer).  J and the operator outputs equal
    those of marching every CTA bit for bit: at the headline grid (cascade 6 of 8), on a
    ragged grid whose top probes sit outside the domain, and where the top cascade is the
    plan's last one (b = inf), with 16-bit storage and a partial wavelength block."""
    rcx = _rcx()
    rng = np.random.default_rng(nx * 3 + nz)
    chi = (10 ** rng.uniform(-4, 1.5, (nl, nz, nx))).astype(np.float32)
    eta = (chi * 10 ** rng.uniform(-1, 1, chi.shape)).astype(np.float32)
    dchi, deta = torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda()
    p = rcx.Plan(nx, nz, C, precision=prec)
    top, listed, total = p.top_list()
    assert top >= 1 and 0 <= 2 * listed <= total, (top, listed, total)
    with_list = [t.cpu() for t in p.formal_solve_mali(dchi, deta)]
    p.set_top_list(False)
    every = [t.cpu() for t in p.formal_solve_mali(dchi, deta)]
    p.set_top_list(True)
    again = [t.cpu() for t in p.formal_solve_mali(dchi, deta)]
    p.close()
    for a, b, c in zip(with_list, every, again):
        assert torch.equal(a, b), f"max abs diff {(a - b).abs().max().item():.3e}"
        assert torch.equal(a, c)


def test_no_top_list_where_most_top_rays_reach_the_box():
    """200^2 with 6 cascades: cascade 5 starts beyond every probe's farthest corner, so the
    top launched cascade is 4, whose rays mostly cross the domain: no list is kept and the
    solve marches every CTA (the 1e-3 oracle parity of that plan is the ragged-shape test)."""
    rcx = _rcx()
    p = rcx.Plan(200, 200, 6)
    assert p.top_list() == (-1, 0, 0)
    p.close()


def test_listed_top_cascade_matches_oracle():
    """300 x 260 with 6 cascades: cascade 5 (the plan's last, b = inf) runs over its listed
    CTAs, a small share of them (rays from the corner probes that still reach the domain);
    J within 1e-3 of the oracle, 17 wavelengths (a ragged second block)."""
    rcx = _rcx()
    p = rcx.Plan(300, 260, 6)
    top, listed, total = p.top_list()
    p.close()
    assert top == 5 and 0 < listed and 4 * listed < total, (top, listed, total)
    chi, eta = W.grf_fields(300, 17, nz=260)
    J = _solve(chi, eta, 6)
    _assert_close(J, _oracle(chi, eta, 6), 1e-3, "J 300x260, listed top cascade")
