"""The C-ABI library builds for sm_103a and exports every entry point that
include/kfbi.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "kfbi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kfbi_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_all_declared_symbols():
    from paper_2309_05965_gb300 import build, kfbi
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers every declared entry point
    covered = set(kfbi.SIGNATURES) | {"kfbi_last_error", "kfbi_mlp_last_error"}
    assert set(names) <= covered, set(names) - covered


def test_binding_refuses_missing_library(tmp_path):
    from paper_2309_05965_gb300 import kfbi
    import pytest
    saved = kfbi._lib
    kfbi._lib = None
    try:
        with pytest.raises(RuntimeError):
            kfbi.load(str(tmp_path / "nope.so"))
    finally:
        kfbi._lib = saved


def test_create_without_gpu_fails_cleanly():
    """Without a CUDA device the library reports an error instead of computing."""
    import torch
    if torch.cuda.is_available():
        return
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    lib = kfbi.load()
    cfg = kfbi.Config(dim=2, n=64, lo=-1.0, hi=1.0, order=4, kind=0, sigma_in=1.0,
                      sigma_out=1.0, kappa=0.0, box_solver=0, precision=0)
    ls = kfbi.LevelSet(kind=1, n_params=5)
    for i, v in enumerate([0.0, 0.0, 0.6, 0.4, 0.0]):
        ls.p[i] = v
    h = ctypes.c_void_p()
    st = lib.kfbi_create_problem(ctypes.byref(cfg), ctypes.byref(ls), None, ctypes.byref(h))
    assert st != 0 and not h.value
