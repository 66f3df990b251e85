"""CPU checks of the C ABI: the library builds for sm_103a, loads without a
GPU and exports every entry point that include/bmdca.h declares; the Python
binding covers the same set of names."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
HEADERS = sorted((ROOT / "include").glob("*.h"))


def declared_functions():
    names = []
    for hdr in HEADERS:
        text = hdr.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(?:int|const char\s*\*)\s*\b(bm_\w+)\s*\(", text):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2501_18456_gb300 import _build
    return _build.build()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for required in ["bm_potts_load", "bm_chains_init", "bm_gibbs_sweep", "bm_chain_stats",
                     "bm_update", "bm_energy_score", "bm_mutant_scan", "bm_seq_weights",
                     "bm_data_stats", "bm_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(str(built_lib))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2501_18456_gb300 import bmdca
    assert set(declared_functions()) <= set(bmdca.SIGNATURES)


def test_version_and_error_calls_need_no_gpu(built_lib):
    lib = ctypes.CDLL(str(built_lib))
    lib.bm_version.restype = ctypes.c_char_p
    lib.bm_last_error.restype = ctypes.c_char_p
    assert lib.bm_version().decode().startswith("bmdca-gb300")
    # argument validation happens before any CUDA call
    lib.bm_potts_load.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] * 3 + [ctypes.c_void_p] * 2
    out = ctypes.c_void_p()
    rc = lib.bm_potts_load(None, None, 4, 21, 0, None, ctypes.byref(out))
    assert rc == -1 and b"NULL" in lib.bm_last_error()
    buf = (ctypes.c_float * 8)()
    rc = lib.bm_potts_load(buf, buf, 4, 33, 0, None, ctypes.byref(out))
    assert rc == -1 and b"q=33" in lib.bm_last_error()


def test_kernel_sources_target_sm103a_only():
    from paper_2501_18456_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
