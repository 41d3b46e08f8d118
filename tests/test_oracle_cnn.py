"""Pins of the oracle's FP64 CNN: convolution special cases, finite-difference
gradients, and one Adam step against its closed form."""
import numpy as np
import pytest

from oracle import cnn


def params(seed, scale=0.3):
    off, n = cnn.offsets()
    rng = np.random.default_rng(seed)
    layers = []
    for cin in cnn.CIN:
        layers.append((rng.normal(0, scale / np.sqrt(9 * cin), (32, 3, 3, cin)), rng.normal(0, 0.05, 32)))
    return cnn.pack(layers, rng.normal(0, 0.3, 32), 0.1)


def test_pack_unpack_layout():
    p = params(0)
    layers, v, c = cnn.unpack(p)
    off, n = cnn.offsets()
    assert n == 32 * (80 + 3 * 304) + 33
    # W_0[o][k]: k = (3 ky + kx) * 8 + c, bias at 72, zeros to 80
    m0 = p[:32 * 80].reshape(32, 80)
    assert m0[5, (3 * 2 + 1) * 8 + 3] == layers[0][0][5, 2, 1, 3]
    assert m0[7, 72] == layers[0][1][7]
    assert np.all(m0[:, 73:] == 0)
    assert np.array_equal(cnn.pack(layers, v, c), p)


def test_conv_identity_kernel_and_shift():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 7, 4))
    w = np.zeros((4, 3, 3, 4))
    for o in range(4):
        w[o, 1, 1, o] = 1.0
    assert np.allclose(cnn.conv3x3(x, w, np.zeros(4)), x)
    # a tap at (ky, kx) = (1, 2) reads the right neighbour; zero padding at the edge
    w = np.zeros((1, 3, 3, 4))
    w[0, 1, 2, 2] = 1.0
    out = cnn.conv3x3(x, w, np.array([0.5]))
    assert np.allclose(out[..., :-1, 0], x[..., 1:, 2] + 0.5)
    assert np.allclose(out[..., -1, 0], 0.5)
    # translation equivariance away from the boundary
    wr = rng.normal(size=(3, 3, 3, 4))
    a = cnn.conv3x3(x, wr, np.zeros(3))
    b = cnn.conv3x3(np.roll(x, 1, axis=2), wr, np.zeros(3))
    assert np.allclose(a[:, :, 1:5], b[:, :, 2:6])


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_by_central_differences(seed):
    rng = np.random.default_rng(seed + 10)
    x = rng.normal(size=(3, 4, 6, 8))
    x[..., 3:] = 0.0
    y = rng.normal(size=3)
    p = params(seed)
    loss, g = cnn.loss_and_grad(p, x, y)
    off, n = cnn.offsets()
    # probe every bias, head entry and a sample of weights of every layer
    idx = list(range(off[4], n))
    for l, (cin, kp) in enumerate(zip(cnn.CIN, cnn.KPAD)):
        m = np.arange(32 * kp).reshape(32, kp) + off[l]
        idx += list(m[:, 9 * cin])
        idx += list(rng.choice(m[:, :9 * min(cin, 3) if l == 0 else 9 * cin].ravel(), 12, replace=False))
    def fd(i, h):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        return (cnn.loss_and_grad(pp, x, y)[0] - cnn.loss_and_grad(pm, x, y)[0]) / (2 * h)

    for i in idx:
        d = fd(i, 1e-6)
        if abs(d - g[i]) > 1e-6 * max(1.0, abs(d)):
            # a ReLU kink within the step: shrink it below the nearest kink
            d = fd(i, 1e-8)
            assert abs(d - g[i]) <= 1e-5 * max(1.0, abs(d)), (i, d, g[i])
    # padding columns and unused input channels carry no gradient
    for l, (cin, kp) in enumerate(zip(cnn.CIN, cnn.KPAD)):
        m = g[off[l]:off[l] + 32 * kp].reshape(32, kp)
        assert np.all(m[:, 9 * cin + 1:] == 0)


def test_adam_first_step_moves_by_lr():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 0.0])
    opt = cnn.Adam(3, lr=0.01)
    q = opt.step(p, g)
    # bias-corrected first step: lr * g / (|g| + eps)
    assert np.allclose(q, p - 0.01 * g / (np.abs(g) + 1e-8))


@pytest.mark.parametrize("nx,ny,factor", [(13, 10, 4), (16, 8, 4), (513, 129, 4)])
def test_fields_block_means_on_ragged_lattices(nx, ny, factor):
    """network input of a constructed equilibrium state (numpy f^eq, no force,
    so rho and u are those of the construction) against block means taken by
    loops: blocks tile the lattice from node (0, 0); rows and columns past the
    last whole block (here the top row and outlet column of 513 x 129) are not
    in the input"""
    import oracle as orc
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    rho = 1.0 + 1e-3 * np.sin(0.7 * X) + 2e-3 * np.cos(0.3 * Y)
    ux = 0.01 * np.cos(0.2 * X + 0.1 * Y)
    uy = -0.005 * np.sin(0.5 * Y) + 1e-4 * X
    cu = cx[:, None, None] * ux + cy[:, None, None] * uy
    f = w[:, None, None] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy))
    c = orc.cfg(nx, ny, tau=0.6)
    got = cnn.fields(c, f, factor, 1000.0, 50.0)
    H, W = ny // factor, nx // factor
    assert got.shape == (H, W, 8)
    for by in range(H):
        for bx in range(W):
            cells = [(y, x) for y in range(by * factor, (by + 1) * factor) for x in range(bx * factor, (bx + 1) * factor)]
            want = [1000.0 * np.mean([rho[y, x] - 1.0 for y, x in cells]),
                    50.0 * np.mean([ux[y, x] for y, x in cells]),
                    50.0 * np.mean([uy[y, x] for y, x in cells])]
            assert np.allclose(got[by, bx, :3], want, rtol=1e-10, atol=1e-13), (by, bx)
    assert np.all(got[..., 3:] == 0)
