"""Batched formal solutions (one launch per cascade over a cost-sorted work list, or a
domain's own launch sequence when it fills the GPU alone,
captured in a CUDA graph) against the per-domain path and the FP64 oracle, with FP32,
FP16 and BF16 interval storage, and the lane-layout autotuners."""
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


def _close(J, J_ref, rtol, what):
    J = np.asarray(J, np.float64)
    floor = 1e-7 * np.abs(J_ref).max()
    bad = np.abs(J - J_ref) > rtol * np.abs(J_ref) + floor
    assert not bad.any(), f"{what}: {bad.sum()} cells off, max rel " \
                          f"{(np.abs(J - J_ref) / np.maximum(np.abs(J_ref), 1e-300)).max():.2e}"


DOMAINS = [(64, 64, 5), (96, 80, 9), (128, 128, 17), (40, 72, 3)]


def _batch_inputs(domains, C, seed_base=0, **plan_kw):
    rcx = _rcx()
    plans, chis, etas, Js, host = [], [], [], [], []
    for d, (nx, nz, nl) in enumerate(domains):
        chi, eta = W.grf_fields(nx, nl, nz=nz, seed_base=seed_base + 100_000 * (d + 1))
        host.append((chi, eta))
        plans.append(rcx.Plan(nx, nz, C, **plan_kw))
        chis.append(torch.from_numpy(chi).cuda())
        etas.append(torch.from_numpy(eta).cuda())
        Js.append(torch.full_like(chis[-1], float("nan")))
    return rcx, plans, chis, etas, Js, host


@pytest.mark.parametrize("prec", ["f32", "bf16", "f16"])
def test_batch_matches_single_domain_path_and_oracle(prec):
    rcx, plans, chis, etas, Js, host = _batch_inputs(DOMAINS, 6, precision=prec)
    batch = rcx.Batch(plans, chis, etas, Js)
    batch.run()
    torch.cuda.synchronize()
    info = batch.info()
    assert info["launches"] >= 7          # pack + one launch per cascade (+ scales if 16-bit)
    for d, ((chi, eta), p) in enumerate(zip(host, plans)):
        J_single = p.formal_solve(chis[d], etas[d]).cpu().numpy()
        np.testing.assert_array_equal(Js[d].cpu().numpy(), J_single)
        lam = chi.shape[0] - 1
        J_ref, _, _ = oracle.rc_solve(chi[lam].astype(np.float64), eta[lam].astype(np.float64), 6)
        _close(Js[d][lam].cpu().numpy(), J_ref, 1e-3 if prec == "f32" else 5e-3,
               f"{prec} domain {d}")
    batch.close()


def test_solo_and_shared_domains_in_one_graph():
    """A 384^2 domain with 48 wavelengths fills the GPU alone in every cascade (2304 to 9216
    CTAs per wavelength block), so it keeps its own launch sequence inside the graph; the
    three small domains share the per-cascade launches.  Every domain equals its single
    solve bit for bit, and the solo domain matches the oracle."""
    doms = [(384, 384, 48), (64, 64, 5), (96, 80, 9), (40, 72, 3)]
    rcx, plans, chis, etas, Js, host = _batch_inputs(doms, 6)
    batch = rcx.Batch(plans, chis, etas, Js)
    batch.run()
    torch.cuda.synchronize()
    assert batch.info()["solo_domains"] == 1
    for d, p in enumerate(plans):
        np.testing.assert_array_equal(Js[d].cpu().numpy(), p.formal_solve(chis[d], etas[d]).cpu().numpy())
    chi, eta = host[0]
    J_ref, _, _ = oracle.rc_solve(chi[47].astype(np.float64), eta[47].astype(np.float64), 6)
    _close(Js[0][47].cpu().numpy(), J_ref, 1e-3, "solo domain")
    batch.close()


def test_graph_replay_reads_the_bound_buffers():
    rcx, plans, chis, etas, Js, host = _batch_inputs(DOMAINS[:2], 5)
    batch = rcx.Batch(plans, chis, etas, Js)
    batch.run()
    torch.cuda.synchronize()
    first = [j.clone() for j in Js]
    batch.run()
    torch.cuda.synchronize()
    for a, b in zip(first, Js):
        assert torch.equal(a, b)
    for e in etas:
        e.mul_(2.0)                          # J is linear in eta
    batch.run()
    torch.cuda.synchronize()
    for a, b in zip(first, Js):
        torch.testing.assert_close(b, 2.0 * a, rtol=1e-6, atol=0)


def test_batch_autotune_keeps_results():
    rcx, plans, chis, etas, Js, host = _batch_inputs(DOMAINS, 5)
    batch = rcx.Batch(plans, chis, etas, Js, autotune=True)
    batch.run()
    torch.cuda.synchronize()
    info = batch.info()
    assert (info["lambda_block"], info["lambda_per_lane"]) in [(16, 4), (8, 4), (32, 4), (8, 2),
                                                               (4, 4)]
    for d, p in enumerate(plans):
        assert p.lane_layout() == (info["lambda_block"], info["lambda_per_lane"])
        np.testing.assert_array_equal(Js[d].cpu().numpy(), p.formal_solve(chis[d], etas[d]).cpu().numpy())


def test_plan_autotune():
    rcx = _rcx()
    chi, eta = W.grf_fields(96, 11)
    p = rcx.Plan(96, 96, 6)
    dchi, deta = torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda()
    J0 = p.formal_solve(dchi, deta).clone()
    J = torch.empty_like(dchi)
    lb, vl = p.autotune(dchi, deta, J)
    assert p.lane_layout() == (lb, vl)
    assert lb <= 32 and vl <= lb
    np.testing.assert_array_equal(p.formal_solve(dchi, deta).cpu().numpy(), J0.cpu().numpy())


def test_batch_rejects_mismatched_plans():
    rcx = _rcx()
    a = rcx.Plan(32, 32, 5)
    b = rcx.Plan(32, 32, 4)
    x = torch.ones((2, 32, 32), device="cuda")
    with pytest.raises(rcx.RcError):
        rcx.Batch([a, b], [x, x], [x, x], [x.clone(), x.clone()])


def test_uneven_domain_workload_full_size_sampled():
    """The 16-domain workload (sides 256..2048, 32..128 wavelengths, seed 7) in one batch
    with BF16 interval storage; one wavelength of the two smallest domains against the oracle,
    and the largest domain against its own single-domain solve."""
    rcx = _rcx()
    doms = W.batched_domains()
    plans, chis, etas, Js, host = [], [], [], [], []
    for side, nl, sb in doms:
        chi, eta = W.grf_fields(side, nl, seed_base=sb)
        host.append((chi[:1].copy(), eta[:1].copy()))
        plans.append(rcx.Plan(side, side, 8, precision="bf16"))
        chis.append(torch.from_numpy(chi).cuda())
        etas.append(torch.from_numpy(eta).cuda())
        Js.append(torch.empty_like(chis[-1]))
        del chi, eta
    batch = rcx.Batch(plans, chis, etas, Js)
    batch.run()
    torch.cuda.synchronize()
    order = np.argsort([s for s, _, _ in doms])[:2]
    for d in order:
        chi, eta = host[d]
        J_ref, _, _ = oracle.rc_solve(chi[0].astype(np.float64), eta[0].astype(np.float64), 8)
        _close(Js[d][0].cpu().numpy(), J_ref, 5e-3, f"domain {d} ({doms[d][0]}^2)")
    for j in Js:
        assert bool(torch.isfinite(j).all())
    # the largest domain (its long cascades strip-split inside the graph) equals the same
    # plan solved on its own
    big = int(np.argmax([s for s, _, _ in doms]))
    J_single = plans[big].formal_solve(chis[big], etas[big])
    torch.cuda.synchronize()
    assert torch.equal(J_single, Js[big]), float((J_single - Js[big]).abs().max())
    batch.close()


def test_plan_autotune_chooses_the_march_per_cascade():
    """rc_plan_autotune times every cascade with both marches and keeps the faster one per
    cascade (RC_MARCH_TUNED); the choice changes timing only, so J is bit-identical to the
    default plan's."""
    rcx = _rcx()
    chi, eta = W.grf_fields(256, 32)
    dchi, deta = torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda()
    ref = rcx.Plan(256, 256, 7).formal_solve(dchi, deta).cpu()
    plan = rcx.Plan(256, 256, 7)
    J = torch.empty_like(dchi)
    lb, vl = plan.autotune(dchi, deta, J)
    if (lb, vl) == (16, 4):
        assert plan.march() == rcx.Plan.MARCH_TUNED
        assert set(plan.march_cascades()) <= set(range(1, 7))
    J2 = plan.formal_solve(dchi, deta).cpu()
    assert torch.equal(J2, ref) or (lb, vl) != (16, 4)
    if (lb, vl) != (16, 4):      # another layout: same results within the parity tolerance
        assert float(((J2 - ref).abs() / ref.abs().clamp_min(1e-30)).max()) < 1e-5
