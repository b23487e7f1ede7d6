"""The C ABI library builds, loads and exports every declared symbol; host-side
argument checks answer without touching a GPU.  CPU only."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libopta():
    from paper_1407_3535_gb300 import build
    build.build()
    from paper_1407_3535_gb300 import _lib
    return _lib.lib()


def _declared_functions():
    names = []
    for h in ("opta.h", "opta_debug.h", "opta_serve.h"):
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             txt, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_every_declared_symbol_is_exported(libopta):
    from paper_1407_3535_gb300 import _lib
    names = _declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(libopta, n), n
        assert n in _lib.SIGNATURES, n
    assert set(_lib.SIGNATURES) == set(names)


def test_params_default_and_status_strings(libopta):
    import paper_1407_3535_gb300 as opta
    p = opta.opta_params_default()
    assert p.rho_th == pytest.approx(0.8) and p.rho_max == pytest.approx(0.95)
    assert p.xi == pytest.approx(0.005) and p.block == 64 and p.h_max == 9
    assert list(p.sigma_levels)[:p.n_levels] == [0.5, 1.0, 2.0, 3.0]
    for code in range(8):
        s = libopta.opta_status_str(code)
        assert s and len(s) > 1
    assert libopta.opta_status_str(99) == b"unknown status"


def test_invalid_arguments_are_rejected_on_the_host(libopta):
    from paper_1407_3535_gb300 import _lib
    out = ctypes.c_void_p(0)
    # null image
    assert libopta.optA_prepare(None, None, None, 0, None, ctypes.byref(out)) == 1
    # negative size count / bad stride
    img = _lib.OptaImage(10, 10, 5, 0, 0, 1234)
    assert libopta.optA_prepare(ctypes.byref(img), None, None, 0, None, ctypes.byref(out)) == 1
    # template larger than image (zncc_full checks before any CUDA call)
    img = _lib.OptaImage(10, 10, 10, 0, 0, 1234)
    t = _lib.OptaTemplate(11, 3, 3, 0, 0, 5678)
    res = _lib.OptaResult()
    assert libopta.zncc_full(ctypes.byref(img), ctypes.byref(t), None, ctypes.byref(res), None) == 1
    # bad parameters
    p = _lib.OptaParams()
    libopta.opta_params_default(ctypes.byref(p))
    p.h_max = 4
    assert libopta.optA_prepare(ctypes.byref(img), ctypes.byref(p), None, 0, None, ctypes.byref(out)) == 1
    # destroy accepts NULL; null handle queries fail cleanly
    assert libopta.optA_destroy(None) == 0
    b = ctypes.c_size_t(0)
    assert libopta.optA_memory_bytes(None, ctypes.byref(b)) == 1
    assert libopta.optA_search(None, None, 0, None, None) == 1


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    from paper_1407_3535_gb300 import _lib
    monkeypatch.setattr(_lib, "_LIB", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.lib()
