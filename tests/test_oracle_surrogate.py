"""Pins of the surrogate oracle (oracle/surrogate.py): the circular 3x3
convolution against explicit loops, adjoint identities of every layer's
backward pass, and central finite differences of the whole network's loss."""
import numpy as np
import pytest

from oracle import surrogate as S


def test_conv3x3_against_loops():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    out = S.conv3x3(x, W, b)
    for (n, y, xx, o) in [(0, 0, 0, 0), (1, 4, 5, 3), (0, 2, 3, 1), (1, 0, 5, 2)]:
        want = b[o]
        for ky in range(3):
            for kx in range(3):
                want += W[o, ky, kx] @ x[n, (y + ky - 1) % 5, (xx + kx - 1) % 6]
        assert out[n, y, xx, o] == pytest.approx(want, abs=1e-12)


def test_layer_adjoints():
    """<A x, y> = <x, A^T y> for the linear parts of conv, pool and upsample."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 6, 4, 3))
    W = rng.standard_normal((5, 3, 3, 3))
    y = rng.standard_normal((2, 6, 4, 5))
    dx, _, _ = S.conv3x3_backward(x, W, y)
    assert np.sum(S.conv3x3(x, W, np.zeros(5)) * y) == pytest.approx(np.sum(x * dx), rel=1e-12)
    p = rng.standard_normal((2, 3, 2, 3))
    assert np.sum(S.pool2(x) * p) == pytest.approx(np.sum(x * S.pool2_backward(p)), rel=1e-12)
    u = rng.standard_normal((2, 12, 8, 3))
    assert np.sum(S.up2(x) * u) == pytest.approx(np.sum(x * S.up2_backward(u)), rel=1e-12)


def test_conv_weight_gradient_is_linear_in_input():
    """dL/dW for L = <conv(x), y> is sum_y x(y + d) y(y): check one tap."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 4, 5, 2))
    W = rng.standard_normal((3, 3, 3, 2))
    y = rng.standard_normal((1, 4, 5, 3))
    _, dW, db = S.conv3x3_backward(x, W, y)
    want = np.einsum("bhwo,bhwc->oc", y, np.roll(x, (-1, 1), axis=(1, 2)))   # ky=2 (dy=+1), kx=0 (dx=-1)
    assert np.allclose(dW[:, 2, 0, :], want, atol=1e-12)
    assert np.allclose(db, y.sum(axis=(0, 1, 2)))


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_network_gradients_by_finite_differences(levels):
    rng = np.random.default_rng(3 + levels)
    net = S.init_net(levels, 4, 3, 2, rng)
    H = 4 << (levels - 1)
    x = rng.standard_normal((2, H, H, 3))
    t = rng.standard_normal((2, H, H, 2))
    L0, dW, db, dWh, dbh = S.backward(net, x, t)
    assert L0 == pytest.approx(S.loss(S.forward(net, x)[0], t))
    eps = 1e-6

    def fd(arr, idx):
        old = arr[idx]
        arr[idx] = old + eps
        lp = S.loss(S.forward(net, x)[0], t)
        arr[idx] = old - eps
        lm = S.loss(S.forward(net, x)[0], t)
        arr[idx] = old
        return (lp - lm) / (2 * eps)

    for k in range(len(net.W)):
        for idx in [(0, 0, 0, 0), (net.W[k].shape[0] - 1, 2, 1, net.W[k].shape[3] - 1), (1, 1, 2, 0)]:
            assert dW[k][idx] == pytest.approx(fd(net.W[k], idx), rel=1e-5, abs=1e-9), (k, idx)
        assert db[k][0] == pytest.approx(fd(net.b[k], (0,)), rel=1e-5, abs=1e-9)
    assert dWh[1, 2] == pytest.approx(fd(net.Wh, (1, 2)), rel=1e-5, abs=1e-9)
    assert dbh[0] == pytest.approx(fd(net.bh, (0,)), rel=1e-5, abs=1e-9)


def test_conv_specs_of_the_paper_surrogate():
    """4 levels, 32 base channels, 8 inputs: 14 convolutions."""
    specs = S.conv_specs(4, 32, 8)
    assert specs[0] == (8, 32) and specs[7] == (256, 256)
    assert specs[8] == (256 + 128, 128) and specs[-1] == (32, 32)
    assert len(specs) == 14
