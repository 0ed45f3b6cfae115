"""Host-side checks of the C-ABI library (no GPU compute).

* libemri.so builds for sm_103a and exports every function include/emri.h
  declares;
* without a usable device every entry point fails with EMRI_ECUDA and a
  message, never a silent fallback;
* the binding refuses to run without the library;
* the product package never imports the oracle (and vice versa).
"""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "emri.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(emri_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2311_17174_gb300 import build as B
    return B.build()


def test_header_declares_the_path_calls():
    names = declared_functions()
    for must in ("emri_ak_waveform", "emri_fft_batch", "emri_loglike_batch", "emri_serve_submit",
                 "emri_serve_poll", "emri_dataset_create", "emri_ctx_create", "emri_autotune",
                 "emri_loglike_multi", "emri_prologue", "emri_stretch_step"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = C.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (emri_[a-z0-9_]+)", out))
    assert set(declared_functions()) <= exported


def test_no_device_fails_loudly(lib_path):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2311_17174_gb300 import emri
    with pytest.raises(emri.EmriError) as ei:
        emri.Context(0)
    assert ei.value.code == emri.ECUDA


def test_context_calls_reject_a_null_context(lib_path):
    """Entry points that take a context check it before touching a device:
    EMRI_EINVAL and a message, with or without a GPU."""
    from paper_2311_17174_gb300 import emri
    lib = emri.load()
    for call in (lambda: lib.emri_ctx_set_pipeline(None, emri.MIXED, 2),
                 lambda: lib.emri_ctx_profile(None, 1),
                 lambda: lib.emri_ctx_launches(None, None)):
        assert call() == emri.EINVAL
        assert lib.emri_last_error()


def test_opts_default_roundtrip(lib_path):
    from paper_2311_17174_gb300 import emri
    o = emri.Opts()
    emri.load().emri_opts_default(C.byref(o))
    assert (o.precision, o.n_max, o.doppler, o.pn_terms, o.mode) == (0, 10, 1, 1, 0)
    assert (o.n_xi, o.omega_m, o.h0) == (2.0, 0.315, 67.4)


def test_missing_library_raises(tmp_path):
    from paper_2311_17174_gb300 import emri
    saved = emri._lib
    emri._lib = None
    try:
        with pytest.raises(RuntimeError):
            emri.load(str(tmp_path / "nope.so"))
    finally:
        emri._lib = saved


def test_product_and_oracle_are_separate():
    pkg = os.path.join(ROOT, "paper_2311_17174_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, flags=re.M), f
                assert "liboracle" not in text and "emri_oracle" not in text, f
    otext = "".join(open(os.path.join(ROOT, "oracle", f)).read()
                    for f in sorted(os.listdir(os.path.join(ROOT, "oracle"))) if f.endswith((".c", ".py")))
    assert "paper_2311_17174_gb300.emri" not in otext and "libemri" not in otext and "emri_common" not in otext
