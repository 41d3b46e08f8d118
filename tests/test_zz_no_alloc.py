"""lbm_step_noalloc, the entry point for callers that cannot allocate device
memory (their device memory belongs to another allocator, or they cannot take
the synchronisation of cudaMalloc): two calls in a row, through the C ABI,
must reproduce two steps of the ensemble API on the same initial state.

Kept in a file of its own that collects last."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

POP_TOL = 1e-5
DRAG_TOL = 1e-4


@pytest.fixture(scope="module")
def L():
    from paper_2005_09323_gb300 import build, lbmrare
    build.build()
    lbmrare.lib()
    return lbmrare


def pack(L, pops, storage, nx, ny):
    """caller-owned buffer [N][9][ny][pitch] holding the given FP64 populations"""
    pitch = L.noalloc_pitch(nx)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    if storage == "fp32":
        buf = torch.zeros((len(pops), 9, ny, pitch), dtype=torch.float32)
        for c, f in enumerate(pops):
            buf[c, :, :, :nx] = torch.from_numpy(f.astype(np.float32))
    else:
        dt = torch.float16 if storage == "fp16" else torch.bfloat16
        buf = torch.zeros((len(pops), 9, ny, pitch), dtype=dt)
        for c, f in enumerate(pops):
            buf[c, :, :, :nx] = torch.from_numpy(f - w).to(dt)
    return buf.cuda()


def unpack(buf, c, storage, nx):
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    a = buf[c, :, :, :nx].float().cpu().numpy().astype(np.float64)
    return a if storage == "fp32" else a + w


@pytest.mark.parametrize("storage,obstacle", [("fp32", (50, 14, 9, 7)), ("fp16", (50, 14, 9, 7)),
                                              ("bf16", (50, 14, 9, 7)), ("fp32", (0, 0, 0, 0)),
                                              ("fp16", (0, 0, 0, 0))])
def test_noalloc_two_steps_match_ensemble(L, storage, obstacle):
    nx, ny, n = 200, 37, 3
    kw = dict(nx=nx, ny=ny, obstacle=obstacle, tau=0.6, gx=2e-5, gy=-5e-6, max_steps=8, storage=storage)
    cfg = L.config(**kw)
    stream = torch.cuda.current_stream()
    e = L.lbm_ensemble_create(cfg, n, 5, stream)
    try:
        pops0 = [L.lbm_ensemble_get_populations(e, c, nx, ny) for c in range(n)]
        L.lbm_ensemble_step(e, 2)
        ref = [L.lbm_ensemble_get_populations(e, c, nx, ny) for c in range(n)]
        ref_drag = np.zeros((n, 2))
        L.lbm_ensemble_drag(e, 0, 2, ref_drag)
    finally:
        L.lbm_ensemble_destroy(e)
    a = pack(L, pops0, storage, nx, ny)
    b = torch.zeros_like(a)
    d1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    d2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    L.lbm_step_noalloc(cfg, n, a, b, d1, stream)
    L.lbm_step_noalloc(cfg, n, b, a, d2, stream)
    torch.cuda.synchronize()
    for c in range(n):
        got = unpack(a, c, storage, nx)
        assert np.abs(got - ref[c]).max() <= POP_TOL * np.abs(ref[c]).max()
    drag = torch.stack([d1, d2], dim=1).cpu().numpy()
    if obstacle[2] == 0:  # no obstacle, no drag
        assert np.all(drag == 0.0) and np.all(ref_drag == 0.0)
    else:
        assert np.abs(drag - ref_drag).max() <= DRAG_TOL * np.abs(ref_drag).max()


def test_noalloc_rejects_oversized_scratch(L):
    """Buffers of the right size and type, so that only the scratch limit can
    reject the call: 1200 clones of 256 x 128 with a 60 x 124 obstacle that
    spans two 128-site row segments need 1200 x (126 rows x 2 segments) drag
    slots x 4 bytes, more than the fixed 1 MiB."""
    n, nx, ny = 1200, 256, 128
    cfg = L.config(nx, ny, obstacle=(100, 2, 60, 124), tau=0.6, max_steps=1)
    a = torch.zeros((n, 9, ny, L.noalloc_pitch(nx)), dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    d = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LbmError) as ei:
        L.lbm_step_noalloc(cfg, n, a, b, d)
    assert ei.value.status == L.LBM_ERR_ARG
    assert "1048576" in str(ei.value)
    del a, b
    torch.cuda.empty_cache()


def test_noalloc_wrapper_rejects_short_or_mistyped_buffers(L):
    nx, ny, n = 64, 16, 2
    cfg = L.config(nx, ny, tau=0.6, max_steps=1, storage="fp16")
    shape = (n, 9, ny, L.noalloc_pitch(nx))
    a = torch.zeros(shape, dtype=torch.float16, device="cuda")
    d = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):  # FP32 buffers for 16-bit storage
        L.lbm_step_noalloc(cfg, n, a.float(), a.float().clone(), d)
    with pytest.raises(TypeError):  # one clone short
        L.lbm_step_noalloc(cfg, n, a[:1].contiguous(), a.clone(), d)
    with pytest.raises(TypeError):  # drag for one clone only
        L.lbm_step_noalloc(cfg, n, a, a.clone(), d[:1])
