"""Pins of the oracle's warm-start network: the reverse-mode gradient equals
central finite differences of the loss (every layer, both boundary kinds);
the convolution matches a brute-force triple loop; its adjoint satisfies
<conv x, g> = <x, conv_adjoint g>."""
import numpy as np
import pytest

from oracle import net


def _brute_conv(x, W, b, periodic):
    C, nz, ny, nx = x.shape
    y = np.zeros((W.shape[0], nz, ny, nx))
    for z in range(nz):
        for yy in range(ny):
            for xx in range(nx):
                for k, (dx, dy, dz) in enumerate(net.OFFSETS):
                    q = [xx + dx, yy + dy, z + dz]
                    ok = True
                    for a, L in enumerate((nx, ny, nz)):
                        if periodic[a]:
                            q[a] %= L
                        elif not 0 <= q[a] < L:
                            ok = False
                    if ok:
                        y[:, z, yy, xx] += W[:, :, k] @ x[:, q[2], q[1], q[0]]
    return y + b[:, None, None, None]


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 1, 0)])
def test_conv_brute_force_and_adjoint(periodic):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 4, 5, 6))
    W = rng.standard_normal((2, 3, 27))
    b = rng.standard_normal(2)
    y = net.conv(x, W, b, periodic)
    assert np.allclose(y, _brute_conv(x, W, b, periodic), atol=1e-12)
    g = rng.standard_normal(y.shape)
    lhs = ((y - b[:, None, None, None]) * g).sum()
    rhs = (x * net.conv_adjoint(g, W, periodic)).sum()
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0)])
def test_gradient_matches_finite_differences(periodic):
    rng = np.random.default_rng(1)
    shape = (4, 5, 6)
    x = rng.standard_normal((2,) + shape)
    t = rng.standard_normal(shape)
    mask = rng.random(shape) < 0.7
    w = net.init_params(3) + 0.05 * rng.standard_normal(net.n_params())
    loss, g = net.loss_grad(x, t, mask, w, periodic)
    idx = rng.choice(net.n_params(), 60, replace=False)
    # include every bias and the last layer
    idx = np.unique(np.concatenate([idx, np.arange(net.n_params() - 5, net.n_params())]))
    h = 1e-6
    for i in idx:
        wp = w.copy(); wp[i] += h
        wm = w.copy(); wm[i] -= h
        fd = (net.loss_grad(x, t, mask, wp, periodic)[0] - net.loss_grad(x, t, mask, wm, periodic)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
