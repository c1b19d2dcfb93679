"""The C-ABI library loads and exports every function include/aerafold.h declares (CPU only:
no compute call is made without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aerafold.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ar_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1507_07733_gb300 import binding
    if not os.path.exists(binding.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build_library()
    return ctypes.CDLL(binding.LIB_PATH)


def test_header_declares_the_abi():
    d = declared()
    for name in ("ar_create", "ar_destroy", "ar_load_pattern", "ar_unfold", "ar_unfold_host", "ar_sync"):
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_1507_07733_gb300 import binding
    assert sorted(binding.EXPORTED) == declared()
    for name in declared():
        assert callable(getattr(binding, name))


def test_status_strings_without_gpu(lib):
    lib.ar_status_string.restype = ctypes.c_char_p
    assert lib.ar_status_string(0) == b"AR_OK"
    assert lib.ar_status_string(9) == b"AR_ERR_DEVICE"


def test_missing_library_fails_loudly(tmp_path):
    from paper_1507_07733_gb300 import binding
    with pytest.raises(binding.LibraryMissing):
        binding._lib = None
        try:
            binding.load(str(tmp_path / "nope.so"))
        finally:
            binding._lib = None
