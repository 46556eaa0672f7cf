"""Host-side checks of the C ABI: the library builds, loads and exports every
entry point declared in include/rlb.h; argument validation that needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rlb_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1211_3286_gb300 import build
    build.build()
    from paper_1211_3286_gb300 import _lib
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    decl = _declared()
    assert len(decl) >= 12
    for name in decl:
        assert hasattr(lib, name), name


def test_binding_covers_declared_symbols():
    from paper_1211_3286_gb300 import _lib
    for name in _declared():
        assert hasattr(_lib, name), name


def _cfg(**kw):
    from paper_1211_3286_gb300 import _lib as L
    c = L.rlb_config()
    c.nx, c.ny, c.nz = kw.get("nx", 8), kw.get("ny", 1), kw.get("nz", 1)
    c.lattice, c.eos = kw.get("lattice", L.RLB_D3Q19), L.RLB_EOS_ULTRAREL
    c.collision = kw.get("collision", L.RLB_MRT)
    c.tau_f, c.tau_v, c.tau_e, c.tau_eps, c.tau_q = kw.get("taus", (0.9, 0.9, 0.55, 0.8, 0.0))
    for a in range(3):
        c.bc[a] = L.RLB_PERIODIC
    c.precision = kw.get("precision", L.RLB_FP64)
    c.correction = kw.get("correction", L.RLB_CORR_NONE)
    return c


@pytest.mark.parametrize("kw, what", [
    (dict(nx=0), "extents"), (dict(lattice=27), "lattice must be"), (dict(lattice=9, nz=2), "D2Q9"),
    (dict(lattice=9, precision=1), "D2Q9"), (dict(collision=7), "collision"),
    (dict(precision=5), "precision"), (dict(taus=(0.5, 0.9, 0.55, 0.8, 0.0)), "tau_f"),
    (dict(taus=(0.9, 0.9, 0.4, 0.8, 0.0)), "tau_e"), (dict(taus=(0.9, 0.9, 0.55, 0.8, 0.3)), "tau_q"),
    (dict(lattice=9, correction=3), "unknown correction"), (dict(correction=1), "needs RLB_D2Q9"),
    (dict(lattice=9, collision=0, correction=2), "needs RLB_D2Q9"),
])
def test_create_rejects_invalid_config_before_touching_the_gpu(lib, kw, what):
    from paper_1211_3286_gb300 import _lib as L
    h = ctypes.c_void_p()
    rc = lib.rlb_create(ctypes.byref(_cfg(**kw)), ctypes.byref(h))
    assert rc == L.RLB_EINVAL
    assert h.value is None
    assert what.lower() in L.rlb_last_error(None).lower()


def test_null_handle_calls_are_rejected(lib):
    from paper_1211_3286_gb300 import _lib as L
    assert lib.rlb_step(None, 1) == L.RLB_EINVAL
    assert lib.rlb_state_bytes(None) == 0
    assert lib.rlb_steps_done(None) == -1
    lib.rlb_destroy(None)
