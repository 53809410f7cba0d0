"""The surrogate's 64 x 64 layer on the tcgen05 tensor cores (bf16 operands in shared
memory, FP32 accumulation in tensor memory) against the FP32-FMA path and the FP64
oracle with h1 rounded to bf16 as the tensor cores see it.  Collected after the other
GPU tests except the allocation-free one."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _problem(B, seed=0):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.3, 4803).astype(np.float32)
    X = rng.normal([4.0, 16.0, 17.0, -12.0, -13.0, -9.0], [0.8, 1.0, 0.9, 1.5, 1.5, 1.5],
                   (B, 6)).astype(np.float32)
    return theta, X, X.mean(axis=0).astype(np.float32), X.std(axis=0).astype(np.float32)


def _oracle_bf16_h1(theta, X, mean, std):
    """FP64 forward with bf16 weights and h1 rounded to bf16 (the MMA's A operand).

    Rounding h1 to bf16 is a discrete decision that the kernel takes on its FP32 value of
    h1.  The FP32 value differs from the FP64 one by at most the FP32 evaluation error of
    the standardisation, the 6-term pre-activation and tanh: bounded here by
    8 * 2^-24 * (|b1| + sum_f |W1_f xn_f|) + 4 * 2^-24 |h1| (a few roundings each, tanhf within
    2 ulps; |tanh'| <= 1).  Where the FP64 h1 lies within that bound of a bf16 rounding
    midpoint either rounding is accepted: the returned slack per sample and output is the
    most one bf16 step of such an h1_j can move y_o, sum_k |W3_ok| |W2_kj| step."""
    W1, b1, W2, b2, W3, b3 = omlp.unflatten(omlp.round_bf16(theta))
    xn = (X.astype(np.float64) - mean.astype(np.float64)) / std.astype(np.float64)
    pre = xn @ W1.T + b1
    h1_64 = np.tanh(pre)
    h1 = omlp.round_bf16(h1_64)
    h2 = np.tanh(h1 @ W2.T + b2)
    u = 2.0 ** -24
    err = 8 * u * (np.abs(b1)[None, :] + np.abs(xn) @ np.abs(W1).T) + 4 * u * np.abs(h1_64)
    # bf16 step at |h1|: 2^(e - 7) for |h1| in [2^e, 2^(e+1))
    mag = np.maximum(np.abs(h1_64), 1e-30)
    step = 2.0 ** (np.floor(np.log2(mag)) - 7)
    frac = mag / step
    ambiguous = np.abs(frac - np.floor(frac) - 0.5) * step <= err
    sens = np.abs(W3) @ np.abs(W2)                        # [out][j]
    slack = (ambiguous * step) @ sens.T                   # [sample][out]
    return h2 @ W3.T + b3, slack


@pytest.mark.parametrize("B", [300, 128 * 37])
def test_tensor_core_forward(B):
    from paper_2408_14425_b300 import build, rcx
    build.build()
    theta, X, mean, std = _problem(B)
    net = rcx.MLP()
    net.set_params(theta, mean, std)
    dX = torch.from_numpy(X).cuda()
    y_fma = net.forward(dX).cpu().numpy()
    net.use_tensor_cores(True)
    y_tc = net.forward(dX).cpu().numpy()
    net.tensor_core_status()
    y_ref, slack = _oracle_bf16_h1(theta, X, mean, std)
    scale = np.abs(y_ref).max()
    # FP32 accumulation of 64 products and FP32 tanh: 1e-3 relative; plus the rounding slack
    err = np.abs(y_tc - y_ref)
    bound = 1e-3 * np.abs(y_ref) + 1e-4 * scale + slack
    bad = np.argwhere(err > bound)
    assert bad.size == 0, f"{len(bad)} outputs beyond the bound, first {bad[:3].tolist()}: " \
                          f"{err[tuple(bad[0])]} > {bound[tuple(bad[0])]}"
    # the FMA path keeps h1 in FP32: the two differ only by the bf16 rounding of h1
    assert np.abs(y_tc - y_fma).max() < 2e-2 * scale


def test_tensor_core_training_gradient_matches_oracle():
    """The training tile on the tensor cores (h1 W2^T, dh2 W2 and dh2^T h1 as tcgen05 MMAs,
    activations as hi + lo bf16 parts): loss and gradient against the FP64 oracle within the
    tolerance of the FMA path's gradient test."""
    from paper_2408_14425_b300 import build, rcx
    build.build()
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.3, 4803).astype(np.float32)
    X = rng.normal([4.0, 16.0, 17.0, -12.0, -13.0, -9.0], [0.8, 1.0, 0.9, 1.5, 1.5, 1.5],
                   (1000, 6)).astype(np.float32)
    Y = rng.normal(0, 1.0, (1000, 3)).astype(np.float32)
    mean, std = X.mean(axis=0).astype(np.float32), X.std(axis=0).astype(np.float32)
    net = rcx.MLP()
    net.set_params(theta, mean, std)
    net.use_tensor_cores(False, training=True)
    loss, g = net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
    net.tensor_core_status()
    loss_ref, g_ref = omlp.loss_and_grad(omlp.round_bf16(theta), X, Y, mean.astype(np.float64),
                                         std.astype(np.float64))
    assert loss == pytest.approx(loss_ref, rel=1e-5, abs=0)
    g = g.cpu().numpy()
    err = np.abs(g - g_ref)
    assert np.all(err <= 1e-4 * np.abs(g_ref) + 1e-6 * np.abs(g_ref).max()), \
        f"max gradient error {err.max():.3e} (max |g| {np.abs(g_ref).max():.3e})"


def test_tensor_core_training_is_reproducible_and_learns():
    """Adam on the tensor-core training path: two runs from the same seed end with identical
    parameters (fixed-order gradient sum), and the loss falls as on the FMA path."""
    from paper_2408_14425_b300 import build, rcx
    build.build()
    rng = np.random.default_rng(1)
    X = rng.normal(0, 1, (20000, 6)).astype(np.float32)
    Y = np.stack([np.sin(X[:, 0]), np.tanh(X[:, 1] - X[:, 2]), 0.3 * X[:, 3] * X[:, 4]],
                 axis=1).astype(np.float32)
    dX, dY = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    out = []
    for _ in range(2):
        net = rcx.MLP(seed=7)
        net.use_tensor_cores(False, training=True)
        net.fit_normalization(dX)
        l0, _ = net.loss_grad(dX, dY)
        net.train(dX, dY, batch=1024, steps=600, lr=3e-3, record=False)
        l1, _ = net.loss_grad(dX, dY)
        net.tensor_core_status()
        out.append((net.get_params()[0], l0, l1))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][2] < 0.15 * out[0][1]
