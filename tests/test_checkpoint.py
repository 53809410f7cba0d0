"""Checkpoint files of the non-LTE iteration (host logic only): populations, iteration
count, history and network parameters survive a save/load round trip unchanged."""
import numpy as np
import pytest

from paper_2408_14425_b300 import checkpoint


class _FakeNet:
    def __init__(self, theta, mean, std):
        self.p = (theta, mean, std)

    def get_params(self):
        return self.p

    def set_params(self, theta, mean, std):
        self.p = (np.array(theta), np.array(mean), np.array(std))


def test_round_trip(tmp_path):
    rng = np.random.default_rng(3)
    pops = 10.0 ** rng.uniform(5, 18, size=(3, 40 * 30))
    net = _FakeNet(rng.normal(size=4803).astype(np.float32),
                   rng.normal(size=6).astype(np.float32), rng.uniform(1, 2, 6).astype(np.float32))
    f = str(tmp_path / "ck.npz")
    checkpoint.save(f, pops, 17, history=[0.5, 0.1, 0.02], net=net)
    other = _FakeNet(None, None, None)
    p2, it, hist = checkpoint.load(f, net=other)
    np.testing.assert_array_equal(p2, pops)
    assert p2.dtype == np.float64 and it == 17 and hist == [0.5, 0.1, 0.02]
    for a, b in zip(net.p, other.p):
        np.testing.assert_array_equal(a, b)


def test_load_without_network_parameters(tmp_path):
    f = str(tmp_path / "ck.npz")
    checkpoint.save(f, np.ones((3, 4)), 0)
    with pytest.raises(KeyError):
        checkpoint.load(f, net=_FakeNet(None, None, None))
    p, it, hist = checkpoint.load(f)
    assert it == 0 and hist == [] and p.shape == (3, 4)
