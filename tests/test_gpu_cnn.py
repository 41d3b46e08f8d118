"""GPU CNN surrogate (BF16 tensor-core convolutions, FP32 accumulation) against
the FP64 oracle: forward, gradients of every layer, one Adam step, the field
extraction from populations, and a training run that fits a known target.

Tolerances: BF16 activations and data gradients carry 8 significant bits; the
prediction is compared to 1e-2 of its scale, gradients to 3e-2 in relative L2
norm per layer (the oracle sees the same BF16-rounded weights and inputs)."""
import numpy as np
import pytest
import torch

from tests import seeded_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2005_09323_gb300 import build, lbmrare
    build.build()
    lbmrare.lib()
    return lbmrare


def bf16_round(a):
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def seeded(L, m, seed):
    """load seeded parameters into the model; returns them (FP64) for the oracle"""
    p = si.cnn_params(seed)
    L.cnn_set_params(m, p)
    return p.astype(np.float64)


def conv_layers_bf16(p):
    """the GPU multiplies BF16 copies of the conv weights (biases included)"""
    from oracle import cnn
    off, n = cnn.offsets()
    q = np.asarray(p, dtype=np.float64).copy()
    q[:off[4]] = bf16_round(q[:off[4]])
    return q


def inputs(B, H, W, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((B, H, W, 8), dtype=np.float32)
    x[..., :3] = rng.normal(0, 1, (B, H, W, 3))
    xt = torch.tensor(x).to(torch.bfloat16).cuda().contiguous()
    return xt, xt.float().cpu().numpy().astype(np.float64)


@pytest.fixture(params=[0, 1], ids=["tcgen05", "mma_sync"])
def model(L, request):
    """16 x 32 inputs: the hidden layers run on the tensor-core (tcgen05) path
    (128-pixel blocks of 4 rows x 32) or on the mma.sync path"""
    m = L.cnn_create(16, 32, 8, 42)
    L.cnn_set_conv_path(m, request.param)
    m.seeded_params = seeded(L, m, 42)
    yield m
    L.cnn_status(m)
    L.cnn_destroy(m)


@pytest.mark.parametrize("H,W,B", [(8, 32, 3), (16, 64, 2), (8, 256, 2), (32, 16, 1), (8, 128, 3), (64, 256, 2),
                                   (24, 32, 2), (8, 48, 2), (8, 16, 2), (40, 128, 2)])
def test_tensor_core_path_matches_mma_sync(L, H, W, B):
    """The tcgen05 hidden layers against the mma.sync ones on the same model and
    inputs, for every block geometry (128-pixel blocks of 128/W rows, or of one
    row of 128 pixels, several per row) and two shapes it does not support
    (width 48; 8 x 16, whose 128-pixel blocks of 8 rows do not tile the height
    twice): both runs then take the mma.sync path.  Both accumulate the same BF16 products
    in FP32 in different orders and round the activations to BF16, so values
    agree to a few BF16 units in the last place."""
    xt, _ = inputs(B, H, W, 7)
    y = torch.tensor(np.linspace(-1, 1, B), dtype=torch.float32, device="cuda")
    m = L.cnn_create(H, W, B, 3)
    try:
        out = []
        for path in (1, 0):
            L.cnn_set_conv_path(m, path)
            pred = torch.zeros(B, dtype=torch.float32, device="cuda")
            L.cnn_forward(m, xt, pred)
            loss = torch.zeros(1, dtype=torch.float32, device="cuda")
            L.cnn_gradient(m, xt, y, loss)
            L.cnn_status(m)
            out.append((pred.cpu().numpy().astype(np.float64), L.cnn_get_gradient(m).astype(np.float64)))
        (p1, g1), (p0, g0) = out
        assert np.abs(p0 - p1).max() <= 1e-2 * (np.abs(p1).max() + 1e-3), (p0, p1)
        from oracle import cnn
        off, _ = cnn.offsets()
        for l in range(4):
            sl = slice(off[l], off[l + 1])
            assert np.linalg.norm(g0[sl] - g1[sl]) <= 2e-2 * np.linalg.norm(g1[sl]), l
    finally:
        L.cnn_destroy(m)


def test_tensor_core_forward_at_full_size_matches_oracle(L, orc):
    """64 x 256 inputs (the 4x-downsampled 1024 x 256 channel), the shape the
    throughput bench runs: one row of 128 pixels per block, two blocks per row."""
    from oracle import cnn
    m = L.cnn_create(64, 256, 2, 5)
    try:
        p = conv_layers_bf16(seeded(L, m, 5))
        xt, x = inputs(2, 64, 256, 9)
        pred = torch.zeros(2, dtype=torch.float32, device="cuda")
        L.cnn_forward(m, xt, pred)
        L.cnn_status(m)
        ref, _ = cnn.forward(p, x, store=bf16_round)
        got = pred.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-2 * (np.abs(ref).max() + 1e-3), (got, ref)
    finally:
        L.cnn_destroy(m)


def test_tensor_core_gradient_at_full_size_matches_oracle(L, orc):
    """64 x 256 inputs: the hidden layers' forward, data gradients and weight
    gradients all on tcgen05 (the weight gradient reduces over pixels with
    MN-major operands, four bands of 16 rows per image half).  Against the
    oracle with BF16 storage of activations and gradients, 1.5e-2 relative L2
    per layer, and the bias gradients."""
    from oracle import cnn
    m = L.cnn_create(64, 256, 2, 5)
    try:
        p = conv_layers_bf16(seeded(L, m, 6))
        xt, x = inputs(2, 64, 256, 4)
        y = np.array([0.7, -0.4], dtype=np.float32)
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        L.cnn_gradient(m, xt, torch.tensor(y, device="cuda"), loss)
        L.cnn_status(m)
        g = L.cnn_get_gradient(m).astype(np.float64)
        _, ref16 = cnn.loss_and_grad(p, x, y.astype(np.float64), store=bf16_round)
        off, _ = cnn.offsets()
        for l in range(4):
            sl = slice(off[l], off[l + 1])
            assert np.linalg.norm(g[sl] - ref16[sl]) < 1.5e-2 * np.linalg.norm(ref16[sl]), l
        check_taps_and_biases(g, ref16)
    finally:
        L.cnn_destroy(m)


def check_taps_and_biases(g, ref, tol=3e-2):
    """each tap (ky, kx) of each layer's weight gradient and each layer's bias
    gradient within tol in relative L2 norm: an error confined to one tap or
    to the bias column cannot hide under the layer's norm"""
    from oracle import cnn
    off, _ = cnn.offsets()
    for l, (cin, kp) in enumerate(zip(cnn.CIN, cnn.KPAD)):
        G = g[off[l]:off[l + 1]].reshape(32, kp)
        R = ref[off[l]:off[l + 1]].reshape(32, kp)
        for tap in range(9):
            a, b = G[:, tap * cin:(tap + 1) * cin], R[:, tap * cin:(tap + 1) * cin]
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), (l, tap)
        assert np.linalg.norm(G[:, 9 * cin] - R[:, 9 * cin]) <= tol * np.linalg.norm(R[:, 9 * cin]), (l, "bias")
        assert np.all(G[:, 9 * cin + 1:] == 0.0), (l, "padding")


def test_w128_with_several_rows_per_cta_runs_on_mma_sync(L, orc):
    """A 128-pixel-wide input with more output rows than one per CTA (the
    shape of the one recorded GPU fault: 32 x 128, here batch 8) is routed to
    the mma.sync kernels; one output row per CTA (batch 4) keeps tcgen05.  The
    routed gradient matches the oracle, per layer, per tap and per bias"""
    from oracle import cnn
    m = L.cnn_create(32, 128, 8, 5)
    try:
        assert L.cnn_tensor_core_paths(m, 8) == (False, False)
        assert L.cnn_tensor_core_paths(m, 4) == (True, True)
        p = conv_layers_bf16(seeded(L, m, 7))
        xt, x = inputs(8, 32, 128, 12)
        y = np.linspace(-0.6, 0.9, 8).astype(np.float32)
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        L.cnn_gradient(m, xt, torch.tensor(y, device="cuda"), loss)
        L.cnn_status(m)
        g = L.cnn_get_gradient(m).astype(np.float64)
        _, ref16 = cnn.loss_and_grad(p, x, y.astype(np.float64), store=bf16_round)
        off, _ = cnn.offsets()
        for l in range(4):
            sl = slice(off[l], off[l + 1])
            assert np.linalg.norm(g[sl] - ref16[sl]) < 1.5e-2 * np.linalg.norm(ref16[sl]), l
        check_taps_and_biases(g, ref16)
    finally:
        L.cnn_destroy(m)


def test_forward_matches_oracle(L, orc, model):
    from oracle import cnn
    xt, x = inputs(6, 16, 32, 1)
    pred = torch.zeros(6, dtype=torch.float32, device="cuda")
    L.cnn_forward(model, xt, pred)
    p = conv_layers_bf16(model.seeded_params)
    ref, _ = cnn.forward(p, x)
    got = pred.cpu().numpy()
    scale = np.abs(ref).max() + np.abs(ref - ref.mean()).max()
    assert np.abs(got - ref).max() <= 1e-2 * scale, (got, ref)


def test_gradient_matches_oracle(L, orc, model):
    """Gradients of every layer against the oracle in two ways.  (1) The oracle
    with BF16 storage of activations and pre-activation gradients (what the
    kernels store between layers): same values up to FP32 accumulation order
    and rounding ties, 1.5e-2 relative L2 per layer.  (2) Pure FP64: the BF16
    storage error compounds down the backward chain (deeper layers, larger
    error); bound = 2 x the error that the BF16-storage oracle itself has
    against FP64, plus 1e-2."""
    from oracle import cnn
    xt, x = inputs(4, 16, 32, 2)
    y = np.array([0.3, -1.2, 0.8, 0.1], dtype=np.float32)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    L.cnn_gradient(model, xt, torch.tensor(y, device="cuda"), loss)
    g = L.cnn_get_gradient(model).astype(np.float64)
    p = conv_layers_bf16(model.seeded_params)
    ref_loss, ref = cnn.loss_and_grad(p, x, y.astype(np.float64))
    _, ref16 = cnn.loss_and_grad(p, x, y.astype(np.float64), store=bf16_round)
    assert abs(loss.item() - ref_loss) <= 2e-2 * ref_loss
    off, n = cnn.offsets()

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)
    for l in range(4):
        sl = slice(off[l], off[l + 1])
        assert rel(g[sl], ref16[sl]) < 1.5e-2, (l, rel(g[sl], ref16[sl]))
        assert rel(g[sl], ref[sl]) < 2 * rel(ref16[sl], ref[sl]) + 1e-2, (l, rel(g[sl], ref[sl]))
    assert rel(g[off[4]:], ref[off[4]:]) < 1e-2


def test_adam_step_matches_oracle(L, model):
    from oracle import cnn
    xt, _ = inputs(4, 16, 32, 3)
    y = torch.tensor([0.5, 0.0, -0.5, 1.0], device="cuda")
    p0 = model.seeded_params
    L.cnn_gradient(model, xt, y)
    g = L.cnn_get_gradient(model).astype(np.float64)
    L.cnn_adam_step(model, 1e-3)
    p1 = L.cnn_get_params(model).astype(np.float64)
    ref = cnn.Adam(len(p0), 1e-3).step(p0, g)
    assert np.abs(p1 - ref).max() <= 1e-6


def test_training_fits_a_known_target(L, model):
    """Target: a fixed linear functional of the field means; 300 Adam steps on
    fresh random batches bring the loss down by over an order of magnitude."""
    torch.manual_seed(0)
    losses = []
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    for step in range(300):
        x = torch.zeros((8, 16, 32, 8), device="cuda")
        x[..., :3] = torch.randn((8, 16, 32, 3), device="cuda") * 0.5 + torch.randn((8, 1, 1, 3), device="cuda")
        xb = x.to(torch.bfloat16).contiguous()
        m = xb.float().mean(dim=(1, 2))
        y = (m[:, 0] - 0.5 * m[:, 1] + 0.25 * m[:, 2]).contiguous()
        L.cnn_train_step(model, xb, y, 3e-3, loss)
        losses.append(loss.item())
    assert np.mean(losses[-20:]) < 0.1 * np.mean(losses[:20]), (losses[:5], losses[-5:])


@pytest.mark.parametrize("nx,ny,factor", [(128, 32, 4), (136, 32, 3)])
def test_fields_match_oracle(L, orc, nx, ny, factor):
    """block means of the flow fields; at 136 x 32 with factor 3 the last
    column and the last two rows are past the last whole block"""
    from oracle import cnn
    kw = dict(nx=nx, ny=ny, obstacle=(30, 12, 8, 8), tau=0.6, gx=2e-5, max_steps=20)
    cfg = L.config(**kw)
    e = L.lbm_ensemble_create(cfg, 3, 5, torch.cuda.current_stream())
    try:
        L.lbm_ensemble_step(e, 15)
        dst = torch.zeros((2, ny // factor, nx // factor, 8), dtype=torch.bfloat16, device="cuda")
        L.lbm_ensemble_fields(e, [2, 0], factor, 1000.0, 50.0, dst, nx, ny)
        oc = orc.cfg(nx, ny, obstacle=(30, 12, 8, 8), tau=0.6, gx=2e-5)
        for i, c in enumerate([2, 0]):
            f, _ = orc.run(oc, orc.init(oc, 5, c, 0.01), 15)  # the oracle's own state of clone c
            ref = cnn.fields(oc, f, factor, 1000.0, 50.0)
            got = dst[i].float().cpu().numpy()
            for ch in range(3):
                scale = np.abs(ref[..., ch]).max()
                assert np.abs(got[..., ch] - ref[..., ch]).max() <= 1e-2 * scale + 1e-6, ch
            assert np.all(got[..., 3:] == 0)
    finally:
        L.lbm_ensemble_destroy(e)


def test_cnn_argument_errors(L, model):
    with pytest.raises(L.LbmError):
        L.cnn_create(12, 32, 4, 0)  # height not a multiple of 8
    x = torch.zeros((9, 16, 32, 8), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(L.LbmError):  # batch beyond max_batch
        L.cnn_forward(model, x, torch.zeros(9, device="cuda"))
    with pytest.raises(TypeError):  # wrong image size is caught before any launch
        L.cnn_forward(model, torch.zeros((2, 8, 32, 8), dtype=torch.bfloat16, device="cuda"),
                      torch.zeros(2, device="cuda"))
    with pytest.raises(L.LbmError):
        L.cnn_set_conv_path(model, 2)
    bad = si.cnn_params(1)
    bad[5] = np.nan
    with pytest.raises(L.LbmError):
        L.cnn_set_params(model, bad)
