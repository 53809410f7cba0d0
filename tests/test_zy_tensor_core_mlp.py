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


def _fma32(a, b, c):
    """float32 fma: the float64 product of two float32 values is exact; one rounding of
    the sum to float32 (a double rounding only in rare ties)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _oracle_bf16_h1(theta, X, mean, std):
    """FP64 forward with bf16 weights and h1 rounded to bf16 (the MMA's A operand).  The
    rounding of h1 to bf16 is a discrete decision, so it is taken on the kernel's FP32
    pre-activation (normalisation, then one fma per input in order, bias first); tanh of
    it in FP64.  Where that value lies within 3 FP32 ulps of a bf16 rounding midpoint
    (CUDA's tanhf is within 2 ulps) the kernel may round the other way; the returned
    slack per sample and output is the most that moves y_o: one bf16 step of h1_j moves it
    by at most sum_k |W3_ok| |W2_kj| step, as |tanh'| <= 1."""
    W1, b1, W2, b2, W3, b3 = omlp.unflatten(omlp.round_bf16(theta))
    m32, istd32 = mean.astype(np.float32), (np.float32(1.0) / std.astype(np.float32))
    xn = (X.astype(np.float32) - m32) * istd32
    pre = np.broadcast_to(b1.astype(np.float32), (X.shape[0], b1.size)).copy()
    for f in range(X.shape[1]):
        pre = _fma32(W1[:, f].astype(np.float32)[None, :], xn[:, f:f + 1], pre)
    h1_64 = np.tanh(pre.astype(np.float64))
    h1 = omlp.round_bf16(h1_64)
    h2 = np.tanh(h1 @ W2.T + b2)
    # bf16 step at |h1|: 2^(e - 7) for |h1| in [2^e, 2^(e+1))
    mag = np.maximum(np.abs(h1_64), 1e-30)
    step = 2.0 ** (np.floor(np.log2(mag)) - 7)
    frac = mag / step
    ambiguous = np.abs(frac - np.floor(frac) - 0.5) * step < 3 * 2.0 ** -23 * mag
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
