"""The C-ABI library loads and exports every entry point its header declares
(no GPU needed: only host-side argument checks are exercised)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2005_09323_gb300 import build, lbmrare
    build.build()
    return lbmrare


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lbmrare.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["lbm_ensemble_create", "lbm_ensemble_step", "lbm_ensemble_drag", "lbm_ensemble_clone",
                 "lbm_ensemble_destroy", "gktl_select", "ams_select", "gktl_weights", "lbm_ensemble_branch"]:
        assert want in names


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/lbmrare.h but not exported"
    assert set(declared_functions()) <= set(L.EXPORTS) | {"lbm_last_error"}


def test_host_argument_checks_need_no_gpu(L):
    lib = L.lib()
    h = C.c_void_p()
    bad = L.config(100, 16)  # nx not a multiple of 8
    assert lib.lbm_ensemble_create(C.byref(bad), 1, 0, None, C.byref(h)) == L.LBM_ERR_ARG
    assert b"multiple of 8" in lib.lbm_last_error()
    bad = L.config(64, 16, tau=0.5)
    assert lib.lbm_ensemble_create(C.byref(bad), 1, 0, None, C.byref(h)) == L.LBM_ERR_ARG
    bad = L.config(64, 16, obstacle=(0, 4, 4, 4))  # touches the periodic seam
    assert lib.lbm_ensemble_create(C.byref(bad), 1, 0, None, C.byref(h)) == L.LBM_ERR_ARG
    assert lib.gktl_weights(0, None, None, None, None) == L.LBM_ERR_ARG
    assert lib.gktl_select(5000, None, 0, 0, None, None, None) == L.LBM_ERR_ARG
    assert lib.ams_select(0, None, 0, 0, None, None, None, None, None) == L.LBM_ERR_ARG
    assert lib.lbm_ensemble_step(None, 1) == L.LBM_ERR_ARG
    n = C.c_uint64(7)
    assert lib.lbm_ensemble_save(None, None, 0, C.byref(n)) == L.LBM_ERR_ARG
    assert lib.lbm_ensemble_load(None, b"LBMRUN", 6) == L.LBM_ERR_ARG
    assert lib.lbm_ensemble_set_perturbation(None, 1) == L.LBM_ERR_ARG


def test_variant_table(L):
    n = L.lbm_step_variant_count()
    assert n >= 3
    kinds = {L.lbm_step_variant_info(i) for i in range(n)}
    for st in (0, 1, 2):
        assert any(k[0] == st for k in kinds)
    with pytest.raises(L.LbmError):
        L.lbm_step_variant_info(n)


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2005_09323_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "oracle.h" not in src, f


def test_every_entry_point_rejects_null_handles_and_empty_sizes(L):
    """Every exported function that takes a handle, an output pointer or a
    count returns LBM_ERR_ARG with a message for a NULL handle (or a zero
    count, or variant index -1), before it touches the GPU; the functions
    without arguments and the destructors (NULL is a no-op) are left out."""
    lib = L.lib()
    skip = {"lbm_last_error", "lbm_launch_count", "lbm_step_variant_count", "lbm_ensemble_destroy", "cnn_destroy",
            "cnn_param_count"}
    special = {"lbm_step_variant_info": (-1, None, None, None), "lbm_step_variant_kind": (-1,)}
    tried = 0
    for name in L.EXPORTS:
        if name in skip:
            continue
        fn = getattr(lib, name)
        args = special.get(name) or tuple(
            None if t is C.c_void_p else (0.0 if t in (C.c_double, C.c_float) else 0) for t in fn.argtypes)
        assert fn(*args) == L.LBM_ERR_ARG, name
        assert lib.lbm_last_error(), name
        tried += 1
    assert tried == len(L.EXPORTS) - len(skip)
    assert lib.lbm_ensemble_destroy(None) == L.LBM_OK and lib.cnn_destroy(None) == L.LBM_OK
    assert lib.cnn_param_count(None) == -1


def test_noalloc_rejects_misaligned_or_invalid_arguments_before_the_gpu(L):
    """lbm_step_noalloc checks the alignment of the caller's buffers (16 bytes
    for the populations, 8 for the drag), the force and the 16-bit scale
    exponent on the host; the pointers below are never dereferenced."""
    lib = L.lib()
    good = L.config(64, 16, tau=0.6, max_steps=1)
    fin, fout, drag = C.c_void_p(0x10000), C.c_void_p(0x20000), C.c_void_p(0x30000)
    cases = [
        (good, C.c_void_p(0x10004), fout, drag, b"16-byte aligned"),
        (good, fin, C.c_void_p(0x20008), drag, b"16-byte aligned"),
        (good, fin, fout, C.c_void_p(0x30004), b"8-byte aligned"),
        (L.config(64, 16, tau=0.6, gx=float("inf"), max_steps=1), fin, fout, drag, b"force"),
        (L.config(64, 16, tau=0.6, gy=float("nan"), max_steps=1), fin, fout, drag, b"force"),
        (L.config(64, 16, tau=0.6, max_steps=1, storage="fp16", shift_exp=40), fin, fout, drag, b"shift_exp"),
    ]
    for cfg, a, b, d, msg in cases:
        assert lib.lbm_step_noalloc(C.byref(cfg), 1, a, b, d, None) == L.LBM_ERR_ARG
        assert msg in lib.lbm_last_error()
