"""The C-ABI library loads and exports every entry point include/dsanls.h declares
(CPU only: no compute call is made without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def _declared():
    names = set()
    for hdr in HEADERS:
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*[\s\*]+(dsanls_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2009_02845_gb300 import build
    return build.build()


def test_header_declares_the_api():
    names = _declared()
    for required in ("dsanls_create", "dsanls_set_dense", "dsanls_set_csr", "dsanls_step", "dsanls_rel_error",
                     "dsanls_get_factors", "dsanls_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in sorted(_declared()):
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(dsanls_[a-z0-9_]+)", out))
    assert _declared() <= exported


def test_binding_symbol_list_matches_header(libpath):
    import paper_2009_02845_gb300 as pkg
    assert set(pkg.EXPORTED_SYMBOLS) == _declared()
    pkg.lib()


def _prototype_arity():
    """Number of parameters of every dsanls_* prototype in the headers."""
    arity = {}
    for hdr in HEADERS:
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"(dsanls_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text, re.S):
            params = m.group(2).strip()
            arity[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return arity


def test_binding_argument_counts_match_the_prototypes(libpath):
    """Every entry point the binding declares takes as many arguments as its
    prototype in the header (a changed signature cannot go unnoticed on CPU)."""
    import paper_2009_02845_gb300._lib as L
    lib = L.lib()
    arity = _prototype_arity()
    assert set(arity) == _declared()
    checked = 0
    for name, n in sorted(arity.items()):
        fn = getattr(lib, name)
        if fn.argtypes is None:
            continue
        assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
        checked += 1
    assert checked >= 30


def test_default_options_without_gpu(libpath):
    import paper_2009_02845_gb300._lib as L
    o = L.Options()
    assert L.lib().dsanls_default_options(ctypes.byref(o)) == 0
    assert o.power_iters == 32 and o.alpha == 1.0 and o.beta == 1.0 and o.solver == L.PGD
    assert L.lib().dsanls_default_options(None) == L.EINVAL


def test_argument_validation_needs_no_gpu(libpath):
    import paper_2009_02845_gb300._lib as L
    h = ctypes.c_void_p()
    lib = L.lib()
    assert lib.dsanls_create(0, 10, 2, 2, 0, 0, ctypes.byref(h)) == L.EINVAL
    assert lib.dsanls_create(10, 10, 0, 2, 0, 0, ctypes.byref(h)) == L.EINVAL
    assert lib.dsanls_create(10, 10, 129, 2, 0, 0, ctypes.byref(h)) == L.EINVAL
    assert lib.dsanls_create(10, 10, 2, 11, L.SUBSAMPLE, 0, ctypes.byref(h)) == L.EINVAL
    assert lib.dsanls_create(10, 10, 2, 9, L.IDENTITY, 0, ctypes.byref(h)) == L.EINVAL
    assert lib.dsanls_create(10, 10, 2, 2, 7, 0, ctypes.byref(h)) == L.EINVAL
    assert lib.dsanls_create(10, 10, 2, 2, 0, 0, None) == L.EINVAL
    assert lib.dsanls_subsample_indices(0, 0, 0, 10, 11, None, None) == L.EINVAL
    assert lib.dsanls_step(None, 1) == L.EINVAL
    assert isinstance(lib.dsanls_last_error(None), bytes)


def test_binding_refuses_to_run_without_the_library(tmp_path, monkeypatch):
    import paper_2009_02845_gb300._lib as L
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "lib_path", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        L.lib()
