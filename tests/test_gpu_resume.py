"""Run resume through the C ABI: lbm_ensemble_save writes an ensemble's run
state to host bytes and lbm_ensemble_load reads it into a fresh ensemble of
the same configuration, which then continues bit for bit as the saved one
does - populations, drag history, observables, the App. D snapshot bank and
perturbation mode (a perturbed branch after the load) and the AMS checkpoints
(a branch to a time before the save).  Loads that do not fit the ensemble are
rejected and leave it unchanged."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

PERIODIC = dict(nx=64, ny=32, obstacle=(16, 12, 8, 8), tau=0.52, gx=1e-5, max_steps=300, ckpt_stride=40,
                n_snapshots=3, init_amp=0.01)
# ragged open channel with square, grid and sponge (as in the open-channel parity tests)
OPEN = dict(nx=203, ny=37, obstacle=(80, 14, 9, 7), tau=0.56, open_x=1, u_in=0.05, grid=(12, 4, 3, 4),
            sponge_len=30, sponge_tau=0.95, max_steps=300, ckpt_stride=40, n_snapshots=3, init_amp=0.01,
            collision="cm", omega_bulk=1.3, omega_3=0.9, omega_4=1.7)


@pytest.fixture(scope="module")
def L():
    from paper_2005_09323_gb300 import build, lbmrare
    build.build()
    lbmrare.lib()
    return lbmrare


class Ens:
    def __init__(self, L, n, seed=0, **kw):
        self.L, self.n = L, n
        self.cfg = L.config(**kw)
        self.h = L.lbm_ensemble_create(self.cfg, n, seed, torch.cuda.current_stream())

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.L.lbm_ensemble_destroy(self.h)

    def pops(self, c):
        return self.L.lbm_ensemble_get_populations(self.h, c, self.cfg.nx, self.cfg.ny)

    def drag(self, t0, t1):
        d = np.zeros((self.n, t1 - t0))
        self.L.lbm_ensemble_drag(self.h, t0, t1, d)
        return d


def same_state(L, a, b, t):
    assert np.array_equal(L.lbm_ensemble_time(a.h, a.n), L.lbm_ensemble_time(b.h, b.n))
    for c in range(a.n):
        assert np.array_equal(a.pops(c), b.pops(c)), f"clone {c}"
    assert np.array_equal(a.drag(0, t), b.drag(0, t))


def run_history(L, e, observe, centred):
    """steps, an App. D snapshot bank, a cloning step and a perturbed AMS branch:
    the pieces of state a resumed run needs (with the printed or the centred
    perturbation coefficients)"""
    if observe:
        L.lbm_ensemble_set_observables(e.h, True)
    L.lbm_ensemble_set_perturbation(e.h, centred)
    L.lbm_ensemble_step(e.h, 90)
    L.lbm_ensemble_set_snapshots(e.h, [0, 2, 3])
    parent = torch.tensor([0, 0, 2, 1], dtype=torch.int32, device="cuda")
    L.lbm_ensemble_clone(e.h, parent, 0.002, 5, 1)
    L.lbm_ensemble_step(e.h, 40)
    L.lbm_ensemble_branch(e.h, 3, 1, 70, 0.002, 5, 2)
    L.lbm_ensemble_step_clones(e.h, 60, [3])


@pytest.mark.parametrize("kw,storage,observe,centred", [(PERIODIC, "fp32", False, False),
                                                        (PERIODIC, "fp16", False, False),
                                                        (PERIODIC, "bf16", True, False), (OPEN, "fp32", True, True)],
                         ids=["periodic-fp32", "periodic-fp16", "periodic-bf16-observables",
                              "open-cm-fp32-centred-perturbation"])
def test_loaded_ensemble_continues_bitwise(L, kw, storage, observe, centred):
    kw = dict(kw, storage=storage)
    with Ens(L, 4, seed=3, **kw) as a:
        run_history(L, a, observe, centred)
        state = L.lbm_ensemble_save(a.h)
        with Ens(L, 4, seed=99, **kw) as b:
            if observe:
                L.lbm_ensemble_set_observables(b.h, True)
            L.lbm_ensemble_load(b.h, state)
            assert L.lbm_ensemble_save(b.h) == state
            same_state(L, a, b, 130)
            # continue both: plain steps, then a perturbed branch from a checkpoint
            # before the save (checkpoints and snapshot bank restored)
            for e in (a, b):
                L.lbm_ensemble_step(e.h, 70)
                L.lbm_ensemble_branch(e.h, 2, 0, 95, 0.002, 7, 3)
                L.lbm_ensemble_step_clones(e.h, 105, [2])
            same_state(L, a, b, 200)
            if observe:
                oa, ob = np.zeros((4, 200, 4)), np.zeros((4, 200, 4))
                L.lbm_ensemble_observables(a.h, 0, 200, oa)
                L.lbm_ensemble_observables(b.h, 0, 200, ob)
                assert np.array_equal(oa, ob)
            assert np.isfinite(a.drag(0, 200)).all()


def test_load_rejects_states_that_do_not_fit(L):
    with Ens(L, 4, seed=3, **PERIODIC) as a:
        L.lbm_ensemble_step(a.h, 30)
        state = L.lbm_ensemble_save(a.h)
        with Ens(L, 4, seed=8, **PERIODIC) as b:
            L.lbm_ensemble_step(b.h, 10)
            before = [b.pops(c) for c in range(4)]
            bad = [state[:-1], state + b"\0", b"x" + state[1:], state[:100]]
            wrong_version = bytearray(state)
            wrong_version[8] ^= 0xFF
            bad.append(bytes(wrong_version))
            for s in bad:
                with pytest.raises(L.LbmError):
                    L.lbm_ensemble_load(b.h, s)
            with pytest.raises(L.LbmError, match="observables"):
                L.lbm_ensemble_set_observables(b.h, True)
                L.lbm_ensemble_load(b.h, state)
            L.lbm_ensemble_set_observables(b.h, False)
            assert list(L.lbm_ensemble_time(b.h, 4)) == [10] * 4
            for c in range(4):
                assert np.array_equal(b.pops(c), before[c])
        for other in (dict(PERIODIC, tau=0.53), dict(PERIODIC, storage="fp16")):
            with Ens(L, 4, seed=3, **other) as b:
                with pytest.raises(L.LbmError, match="configuration"):
                    L.lbm_ensemble_load(b.h, state)
        with Ens(L, 3, seed=3, **PERIODIC) as b:
            with pytest.raises(L.LbmError, match="clone count"):
                L.lbm_ensemble_load(b.h, state)
