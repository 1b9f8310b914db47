"""Pins for the oracle's warm-start network layers: brute-force loops for the
convolution, finite differences for every gradient, adjoint identities for the
resampling layers, and the bfloat16 rounding against its bit-level definition."""
import numpy as np
import pytest

from oracle import nn


def _conv_brute(x, w, b):
    ci, D, H, W = x.shape
    co = w.shape[0]
    y = np.zeros((co, D, H, W))
    for o in range(co):
        for z in range(D):
            for yy in range(H):
                for xx in range(W):
                    s = b[o]
                    for i in range(ci):
                        for t, (dz, dy, dx) in enumerate(nn.TAPS):
                            zz, y2, x2 = z + dz, yy + dy, xx + dx
                            if 0 <= zz < D and 0 <= y2 < H and 0 <= x2 < W:
                                s += w[o, i, t] * x[i, zz, y2, x2]
                    y[o, z, yy, xx] = s
    return y


def test_conv_matches_brute_force():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 4, 5))
    w = rng.normal(size=(3, 2, 27))
    b = rng.normal(size=3)
    assert np.allclose(nn.conv3d(x, w, b), _conv_brute(x, w, b), atol=1e-12)


def test_conv_gradients_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 3, 4))
    w = rng.normal(size=(2, 2, 27))
    b = rng.normal(size=2)
    gy = rng.normal(size=(2, 3, 3, 4))
    gx, gw, gb = nn.conv3d_backward(x, w, gy)
    f = lambda x_, w_, b_: float(np.sum(gy * nn.conv3d(x_, w_, b_)))
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 1, 3), (0, 1, 2, 2)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        assert (f(xp, w, b) - f(xm, w, b)) / (2 * h) == pytest.approx(gx[idx], rel=1e-6, abs=1e-8)
    for idx in [(0, 0, 13), (1, 1, 0), (1, 0, 26)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        assert (f(x, wp, b) - f(x, wm, b)) / (2 * h) == pytest.approx(gw[idx], rel=1e-6, abs=1e-8)
    assert np.allclose(gb, gy.sum(axis=(1, 2, 3)))


def test_resampling_adjoints():
    rng = np.random.default_rng(2)
    a = rng.normal(size=(3, 4, 6, 8))
    c = rng.normal(size=(3, 2, 3, 4))
    # <pool(a), c> = <a, pool_backward(c)>;  <up(c), a> = <c, up_backward(a)>
    assert np.sum(nn.pool2(a) * c) == pytest.approx(np.sum(a * nn.pool2_backward(c)), rel=1e-12)
    assert np.sum(nn.up2(c) * a) == pytest.approx(np.sum(c * nn.up2_backward(a)), rel=1e-12)
    assert np.allclose(nn.pool2(nn.up2(c)), c)


def test_network_gradients_finite_differences():
    rng = np.random.default_rng(3)
    params = nn.init_params(seed=4, c_in=2, c_out=3, widths=(4, 4, 4, 4))
    x = rng.normal(size=(2, 8, 8, 8))
    gy = rng.normal(size=(3, 8, 8, 8))
    y, cache = nn.forward(params, x, keep=True)
    grads = nn.backward(params, cache, gy)
    h = 1e-6
    for li, idx in [(0, (1, 0, 5)), (5, (2, 3, 13)), (10, (0, 1, 26)), (7, (3, 0, 0))]:
        w = params[li][0]
        old = w[idx]
        w[idx] = old + h
        fp = float(np.sum(gy * nn.forward(params, x)))
        w[idx] = old - h
        fm = float(np.sum(gy * nn.forward(params, x)))
        w[idx] = old
        assert (fp - fm) / (2 * h) == pytest.approx(grads[li][0][idx], rel=1e-5, abs=1e-7)
    # bias of the head
    b = params[10][1]
    b[1] += h
    fp = float(np.sum(gy * nn.forward(params, x)))
    b[1] -= 2 * h
    fm = float(np.sum(gy * nn.forward(params, x)))
    b[1] += h
    assert (fp - fm) / (2 * h) == pytest.approx(grads[10][1][1], rel=1e-6)


def test_bf16_rounding():
    vals = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0, 1e-30])
    r = nn.to_bf16(vals)
    # bf16 keeps 8 significand bits: representable values are exact, others round
    assert r[0] == 1.0
    assert r[1] == 1.0            # 1 + 2^-8: tie between 1 and 1 + 2^-7, to even
    assert r[2] == 1.0078125      # 1 + 1.5 * 2^-8 rounds up to 1 + 2^-7
    assert abs(r[3] - (-3.140625)) < 1e-12
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2 ** -8)
    # ties to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> 1
    assert nn.to_bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert nn.to_bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
