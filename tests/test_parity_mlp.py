"""The surrogate network's CUDA kernels against the FP64 oracle, the seeding kernels
against their closed forms, and what a trained network gains over the LTE start."""
import numpy as np
import pytest

from oracle import mlp as omlp
from oracle import nlte
from paper_2408_14425_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ATOM = W.h3_atom()


def _rcx():
    from paper_2408_14425_b300 import build, rcx
    build.build()
    return rcx


def _net_problem(B=1000, seed=0):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.3, 4803).astype(np.float32)
    X = rng.normal([4.0, 16.0, 17.0, -12.0, -13.0, -9.0], [0.8, 1.0, 0.9, 1.5, 1.5, 1.5],
                   (B, 6)).astype(np.float32)
    Y = rng.normal(0, 1.0, (B, 3)).astype(np.float32)
    mean = X.mean(axis=0).astype(np.float32)
    std = X.std(axis=0).astype(np.float32)
    return theta, X, Y, mean, std


def test_forward_matches_oracle_with_bf16_weights():
    rcx = _rcx()
    theta, X, Y, mean, std = _net_problem(B=777)
    net = rcx.MLP()
    net.set_params(theta, mean, std)
    y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    y_ref, _ = omlp.forward(omlp.round_bf16(theta), X, mean.astype(np.float64), std.astype(np.float64))
    np.testing.assert_allclose(y, y_ref, rtol=1e-4, atol=1e-5 * np.abs(y_ref).max())


def test_loss_and_gradient_match_oracle():
    rcx = _rcx()
    theta, X, Y, mean, std = _net_problem(B=1000)
    net = rcx.MLP()
    net.set_params(theta, mean, std)
    loss, g = net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
    loss_ref, g_ref = omlp.loss_and_grad(omlp.round_bf16(theta), X, Y, mean.astype(np.float64),
                                         std.astype(np.float64))
    assert loss == pytest.approx(loss_ref, rel=1e-5, abs=0)
    g = g.cpu().numpy()
    err = np.abs(g - g_ref)
    assert np.all(err <= 1e-4 * np.abs(g_ref) + 1e-6 * np.abs(g_ref).max()), \
        f"max gradient error {err.max():.3e} (max |g| {np.abs(g_ref).max():.3e})"


def test_normalization_and_params_roundtrip():
    rcx = _rcx()
    theta, X, Y, mean, std = _net_problem(B=5000)
    net = rcx.MLP(seed=3)
    net.fit_normalization(torch.from_numpy(X).cuda())
    th, mu, sd = net.get_params()
    np.testing.assert_allclose(mu, X.astype(np.float64).mean(axis=0), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(sd, X.astype(np.float64).std(axis=0), rtol=1e-5)
    net.set_params(theta)
    np.testing.assert_array_equal(net.get_params()[0], theta)


def test_training_reduces_the_loss():
    rcx = _rcx()
    rng = np.random.default_rng(1)
    X = rng.normal(0, 1, (20000, 6)).astype(np.float32)
    Y = np.stack([np.sin(X[:, 0]), np.tanh(X[:, 1] - X[:, 2]), 0.3 * X[:, 3] * X[:, 4]],
                 axis=1).astype(np.float32)
    net = rcx.MLP(seed=7)
    dX, dY = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    net.fit_normalization(dX)
    l0, _ = net.loss_grad(dX, dY)
    hist = net.train(dX, dY, batch=1024, steps=600, lr=3e-3)
    l1, _ = net.loss_grad(dX, dY)
    assert np.all(np.isfinite(hist))
    assert l1 < 0.15 * l0


def test_training_is_reproducible():
    """The tiles' partial gradients are summed in a fixed order (no atomics), so two nets
    with the same seed trained on the same data end with identical parameters."""
    rcx = _rcx()
    rng = np.random.default_rng(4)
    X = rng.normal(0, 1, (9000, 6)).astype(np.float32)
    Y = np.stack([np.cos(X[:, 0]), X[:, 1] * X[:, 2], np.tanh(X[:, 5])], axis=1).astype(np.float32)
    dX, dY = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    out = []
    for _ in range(2):
        net = rcx.MLP(seed=11)
        net.fit_normalization(dX)
        net.train(dX, dY, batch=2000, steps=200, lr=3e-3, record=False)
        torch.cuda.synchronize()
        out.append(net.get_params()[0])
    np.testing.assert_array_equal(out[0], out[1])


def test_features_targets_and_seed_closed_forms():
    rcx = _rcx()
    atom = rcx.Atom(ATOM)
    T, nH, vox = W.prominence_slab(n=32, half_width=6, blend=2, wander=2)
    dT, dnH = torch.from_numpy(T).cuda(), torch.from_numpy(nH).cuda()
    ne, na, pops = atom.lte(dT, dnH)
    J = torch.from_numpy(np.random.default_rng(2).uniform(1e-14, 1e-9, (63, 32 * 32))
                         .astype(np.float32)).cuda()
    X = rcx.surrogate_features(atom, dT, ne, dnH, J).cpu().numpy()
    Jh = J.cpu().numpy()
    np.testing.assert_allclose(X[:, 0], np.log10(T.ravel()), rtol=1e-6)
    np.testing.assert_allclose(X[:, 1], np.log10(ne.cpu().numpy()), rtol=1e-6)
    np.testing.assert_allclose(X[:, 2], np.log10(nH.ravel()), rtol=1e-6)
    for l in range(3):
        np.testing.assert_allclose(X[:, 3 + l], np.log10(Jh[21 * l + 10]), rtol=1e-5)
    # LTE populations have departure coefficients 1
    Y = rcx.surrogate_targets(atom, dT, na, pops).cpu().numpy()
    assert np.abs(Y).max() < 1e-6
    # a network with constant output c seeds n_i ~ 10^c_i n_i(LTE), renormalised
    net = rcx.MLP()
    th = np.zeros(4803, np.float32)
    c = np.array([0.3, -0.2, 0.1], np.float32)
    th[-3:] = c
    net.set_params(th, np.zeros(6), np.ones(6))
    seeded = pops.clone()
    fb = rcx.surrogate_seed(atom, net, torch.from_numpy(X).cuda(), dT, na, seeded)
    assert fb == 0
    lte = nlte.lte_populations(ATOM, T, na.cpu().numpy())
    expect = lte * (10.0 ** omlp.round_bf16(c))[:, None]      # the kernels use bf16 weights
    expect *= na.cpu().numpy() / expect.sum(axis=0)
    np.testing.assert_allclose(seeded.cpu().numpy(), expect, rtol=1e-6)
    # an unusable output falls back to LTE, cell by cell
    th[-3] = np.nan
    net.set_params(th)
    fb = rcx.surrogate_seed(atom, net, torch.from_numpy(X).cuda(), dT, na, seeded)
    assert fb == 32 * 32
    np.testing.assert_allclose(seeded.cpu().numpy(), lte, rtol=1e-12)


def test_trained_network_saves_iterations():
    """Train on 16 small slabs, then solve a held-out slab from LTE and from the seed:
    the seed converges in fewer iterations to the same populations (within 5e-3)."""
    rcx = _rcx()
    from paper_2408_14425_b300 import surrogate
    atom = rcx.Atom(ATOM)
    n = 48
    Xs, Ys = [], []
    for seed in range(100, 116):
        T, nH, vox = W.prominence_slab(n=n, seed=seed, half_width=10, blend=3, wander=3)
        plan = rcx.Plan(n, n, 5, voxel_size=vox)
        X, Y, _ = surrogate.training_pairs(plan, atom, torch.from_numpy(T).cuda(),
                                           torch.from_numpy(nH).cuda())
        Xs.append(X)
        Ys.append(Y)
    X = torch.cat(Xs)
    Y = torch.cat(Ys)
    net = rcx.MLP(seed=11)
    net.fit_normalization(X)
    net.train(X, Y, batch=2048, steps=1500, lr=2e-3, record=False)
    T, nH, vox = W.prominence_slab(n=n, seed=999, half_width=10, blend=3, wander=3)
    plan = rcx.Plan(n, n, 5, voxel_size=vox)
    dT, dnH = torch.from_numpy(T).cuda(), torch.from_numpy(nH).cuda()
    plain = surrogate.solve(plan, atom, dT, dnH)
    seeded = surrogate.solve(plan, atom, dT, dnH, net=net)
    assert plain["converged"] and seeded["converged"]
    assert seeded["iterations"] < plain["iterations"]
    rel = (seeded["pops"] - plain["pops"]).abs() / plain["pops"].abs()
    assert float(rel.max()) < 5e-3


def test_surrogate_interface_names():
    """rc_surrogate_init / _train_step / _predict are rc_mlp_create, one step of
    rc_mlp_train and rc_mlp_forward: five single steps equal one five-step call (up to the
    summation order of the gradient atomics), and predict equals forward."""
    import ctypes
    from paper_2408_14425_b300 import build, rcx
    build.build()
    L = rcx.load()
    rng = np.random.default_rng(2)
    X = torch.from_numpy(rng.normal(size=(3000, 6)).astype(np.float32)).cuda()
    Y = torch.from_numpy(rng.normal(size=(3000, 3)).astype(np.float32)).cuda()
    a = rcx.MLP(seed=5)
    a.fit_normalization(X)
    a.train(X, Y, batch=512, steps=5, lr=1e-3, record=False)
    h = ctypes.c_void_p()
    assert L.rc_surrogate_init(5, ctypes.byref(h)) == 0
    fp = ctypes.POINTER(ctypes.c_float)
    mean = np.ascontiguousarray(a.get_params()[1])
    std = np.ascontiguousarray(a.get_params()[2])
    assert L.rc_mlp_set_params(h, None, mean.ctypes.data_as(fp), std.ctypes.data_as(fp)) == 0
    loss = ctypes.c_float()
    for _ in range(5):
        assert L.rc_surrogate_train_step(h, X.data_ptr(), Y.data_ptr(), 3000, 512, 1e-3,
                                         ctypes.byref(loss), None) == 0
    th = np.empty(a.n_params, np.float32)
    assert L.rc_mlp_get_params(h, th.ctypes.data_as(fp), None, None) == 0
    np.testing.assert_allclose(th, a.get_params()[0], rtol=1e-4, atol=1e-6)
    assert np.isfinite(loss.value) and loss.value > 0
    y1 = torch.empty((3000, 3), device="cuda")
    assert L.rc_surrogate_predict(h, X.data_ptr(), 3000, y1.data_ptr(), None) == 0
    y2 = torch.empty((3000, 3), device="cuda")
    assert L.rc_mlp_forward(h, X.data_ptr(), 3000, y2.data_ptr(), None) == 0
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    L.rc_mlp_destroy(h)
