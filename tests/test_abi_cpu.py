"""The C-ABI library builds for sm_103a, loads without a GPU, exports every entry point that
include/*.h declares, and its host-only helpers (PPL, adaptive time) agree with the oracle."""
import ctypes
import glob
import json
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"^FO_API\s+[^;(]*?\b(fo_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_05709_gb300 import _lib
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2601_05709_gb300 import _lib, build
    names = _declared()
    assert len(names) >= 30
    out = subprocess.run(["nm", "-D", "--defined-only", build.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (fo_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)
        assert n in _lib.PROTOTYPES, f"{n} has no binding"


def test_library_is_sm103a_only(lib):
    from paper_2601_05709_gb300 import build
    assert ["-gencode", "arch=compute_103a,code=sm_103a"] == build.ARCH


def test_ppl_matches_oracle(lib):
    from oracle.ppl import PPL as OPPL
    from paper_2601_05709_gb300.api import PPL
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "ppl_adaptime.json")))["ppl_constant_C_1p2"]
    g, o = PPL(1), OPPL(1)
    rng = np.random.default_rng(3)
    for i in range(20):
        C = 1.2 if i < 2 else 1.0 + 0.3 * rng.standard_normal()
        lam_g, L_g = g.update([C], 2.5)
        lam_o, L_o = o.update([C], 2.5)
        assert lam_g[0] == pytest.approx(lam_o[0], rel=1e-14, abs=1e-16)
        assert L_g == pytest.approx(L_o, rel=1e-14)
        if i == 0:
            assert lam_g[0] == pytest.approx(gold["lambda1"], rel=1e-15)
        if i == 1:
            assert lam_g[0] == pytest.approx(gold["lambda2"], rel=1e-14)


def test_adaptime_matches_oracle_and_golden(lib):
    from oracle.ppl import adaptime as oada
    from paper_2601_05709_gb300.api import adaptime, run_options
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "ppl_adaptime.json")))["adaptime"]
    for case in gold:
        t, n = adaptime(case["Btt"])
        assert t == pytest.approx(case["t_end"], rel=1e-15) and n == case["nsteps"]
    opts = run_options(dfactor=0.1, lv_time=(1e-3, 0.1), lv_iter=(8, 16))
    for B in np.geomspace(1e-6, 1e4, 57):
        t, n = adaptime(B, opts)
        to, no = oada(B, 0.1, (1e-3, 0.1), (8, 16))
        assert t == pytest.approx(to, rel=1e-15) and n == no


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2601_05709_gb300 import _lib, build
    monkeypatch.setattr(build, "lib_path", lambda: str(tmp_path / "absent.so"))
    monkeypatch.setattr(_lib, "_LIB", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load()


def test_context_without_gpu_reports_error(lib):
    # on a machine without a CUDA device the context call returns an error code, never crashes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    h = ctypes.c_void_p()
    st = lib.fo_ctx_create(0, None, 0, ctypes.byref(h))
    assert st != 0
