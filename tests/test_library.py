"""Host-side checks of the C ABI: it builds, exports every declared symbol, and rejects
bad problems before touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2510_07674_gb300 import build as B
from paper_2510_07674_gb300 import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(spasm_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(libpath):
    out = subprocess.check_output(["nm", "-D", "--defined-only", libpath]).decode()
    exported = set(re.findall(r"\bT (spasm_\w+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    assert declared <= exported, declared - exported


def test_binding_names_match_header(libpath):
    from paper_2510_07674_gb300 import spasm as S
    assert set(S.EXPORTED) == _declared()
    L = S.lib()
    for name in S.EXPORTED:
        assert hasattr(L, name)


def test_create_rejects_bad_sizes_on_host(libpath):
    from paper_2510_07674_gb300 import spasm as S
    wl = scenes.make_problem("tower1", seed=0)
    for bad in ({"W": 2}, {"M": 300}, {"P": 100}, {"N": 40000}, {"K_lin": 0}):
        with pytest.raises(S.SpasmError) as e:
            S.Problem(wl, stream=0, **bad)
        assert e.value.status == -1
    wl17 = scenes.make_problem("tower1", seed=0, B=17)
    with pytest.raises(S.SpasmError):
        S.Problem(wl17, stream=0)
    wl_long = scenes.make_problem("tower10", seed=0, B=16, W=40)
    with pytest.raises(S.SpasmError) as e:
        S.Problem(wl_long, stream=0)
    assert "configurations" in str(e.value)


def test_analytic_ik_mode_checked_on_host(libpath):
    """ik_mode must be 0 or 1, and 1 needs the Franka joint layout; both are refused before
    any device work."""
    from paper_2510_07674_gb300 import spasm as S
    wl = scenes.make_problem("tower1", seed=0)
    with pytest.raises(S.SpasmError) as e:
        S.Problem(wl, stream=0, ik_mode=2)
    assert e.value.status == -1 and "ik_mode" in str(e.value)
    bent = scenes.make_problem("tower1", seed=0, ik_mode=1)
    bent.robot.dh[2, 0] = 0.02
    with pytest.raises(S.SpasmError) as e:
        S.Problem(bent, stream=0)
    assert e.value.status == -1 and "Franka" in str(e.value)


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    from paper_2510_07674_gb300 import spasm as S
    monkeypatch.setattr(S, "_lib", None)
    monkeypatch.setattr(S, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        S.lib()
