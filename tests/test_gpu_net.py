"""Warm-start network kernels (BF16 tensor-core implicit GEMMs, FP32
accumulation) against the FP64 numpy oracle: forward output, loss and every
parameter gradient within BF16-level tolerances, on both tensor paths of the
16 -> 16 layers (tcgen05 with the accumulator in tensor memory, and the
warp-level mma.sync form), the two paths against each other, and GPU
training lowers the loss on a learnable mapping."""
import numpy as np
import pytest

import paper_1710_09421_gb300 as E
from oracle import net

pytestmark = pytest.mark.gpu


def _case(seed, shape=(12, 10, 14)):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((2,) + shape).astype(np.float32)
    w = (net.init_params(seed) + 0.02 * rng.standard_normal(net.n_params())).astype(np.float32)
    return rng, x, w


@pytest.fixture(params=[1, 0], ids=["tcgen05", "mma_sync"])
def tensor_path(request):
    lib = E.load()
    prev = lib.ekl_net_tensor_path(request.param)
    yield request.param
    lib.ekl_net_tensor_path(prev)


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (1, 0, 1)])
def test_forward_matches_oracle(periodic, tensor_path):
    rng, x, w = _case(0)
    nz, ny, nx = x.shape[1:]
    y = E.ekl_net_eval((nx, ny, nz), periodic, x, w)
    ref = net.forward(x.astype(np.float64), w.astype(np.float64), periodic)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    print(tensor_path, periodic, err)
    assert err < 1e-2


def test_tcgen05_matches_mma_sync_on_a_ragged_grid():
    """1190 nodes: nine full 128-node tiles and a ragged one.  The two paths
    differ only in the order of the FP32 accumulation inside an MMA, which
    can move a BF16 activation by one unit between layers."""
    rng, x, w = _case(3, (7, 10, 17))
    nz, ny, nx = x.shape[1:]
    lib = E.load()
    prev = lib.ekl_net_tensor_path(1)
    y1 = E.ekl_net_eval((nx, ny, nz), (1, 0, 1), x, w)
    lib.ekl_net_tensor_path(0)
    y0 = E.ekl_net_eval((nx, ny, nz), (1, 0, 1), x, w)
    lib.ekl_net_tensor_path(prev)
    d = np.linalg.norm(y1 - y0) / np.linalg.norm(y0)
    print("tcgen05 vs mma.sync", d)
    assert d < 5e-3


def test_loss_and_gradient_match_oracle(tensor_path):
    rng, x, w = _case(1)
    nz, ny, nx = x.shape[1:]
    t = rng.standard_normal(x.shape[1:]).astype(np.float32)
    mask = (rng.random(x.shape[1:]) < 0.8).astype(np.uint8)
    loss, g = E.ekl_net_loss_grad((nx, ny, nz), (1, 1, 1), x, t, mask, w)
    lref, gref = net.loss_grad(x.astype(np.float64), t.astype(np.float64), mask,
                               w.astype(np.float64), (1, 1, 1))
    assert abs(loss - lref) / lref < 2e-2
    # per layer: W then b.  Every layer's activations and back-propagated
    # gradients are BF16 (8 significant bits, rounding 2^-9): the first
    # layer's gradient has passed three of those roundings (measured 3.1 %
    # off the FP64 oracle), the others at most two (within 1.2 %).
    o = 0
    for layer, (ci, co) in enumerate(zip(net.CHANNELS[:-1], net.CHANNELS[1:])):
        tol = 4e-2 if layer == 0 else 2e-2
        for n in (co * ci * 27, co):
            seg, ref = g[o:o + n], gref[o:o + n]
            print(tensor_path, ci, co, n, np.linalg.norm(seg - ref) / np.linalg.norm(ref))
            assert np.linalg.norm(seg - ref) <= tol * np.linalg.norm(ref) + 1e-7, (ci, co, n)
            o += n


def test_training_lowers_loss():
    """Learn a fixed random network's mapping from its own outputs."""
    rng, _, w_true = _case(2, (16, 16, 16))
    S = 12
    xs = rng.standard_normal((S, 2, 16, 16, 16)).astype(np.float32)
    ts = np.stack([net.forward(xs[s].astype(np.float64), w_true.astype(np.float64), (0, 0, 0))
                   for s in range(S)]).astype(np.float32)
    mask = np.zeros((16, 16, 16), np.uint8)
    mask[4:-4, 4:-4, 4:-4] = 1
    w0 = net.init_params(7).astype(np.float32)
    w1, curve = E.ekl_net_train((16, 16, 16), xs, ts, mask, w0, iters=150, batch=4, lr=3e-3, seed=1)
    assert np.isfinite(curve).all()
    assert curve[-10:].mean() < 0.5 * curve[:10].mean(), (curve[:5], curve[-5:])
