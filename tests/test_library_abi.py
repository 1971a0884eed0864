"""The C-ABI library builds for sm_103a, loads, and exports every function the header declares.

CPU only: nothing here calls into CUDA (only lbm_abi_version / lbm_last_error, which do not).
"""
import ctypes

import pytest

from paper_2512_16230_gb300 import build as B
from paper_2512_16230_gb300 import lbm


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_library_exports_every_declared_function(libpath):
    raw = ctypes.CDLL(libpath)
    declared = lbm.header_functions()
    assert len(declared) >= 20
    missing = [name for name in declared if not hasattr(raw, name)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    assert sorted(lbm.SIGNATURES) == lbm.header_functions()


def test_abi_version_and_error_string(libpath):
    lb = lbm.load(libpath)
    assert lb.lbm_abi_version() == 1
    assert isinstance(lb.lbm_last_error(), bytes)


def test_missing_library_fails_loudly(tmp_path):
    saved = lbm._lib
    lbm._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            lbm.load(str(tmp_path / "nope.so"))
    finally:
        lbm._lib = saved


def _header_enum(name):
    """name -> value of the enumerators of the C typedef enum ``name`` in the header."""
    import re
    text = open(lbm.HEADER).read()
    body = re.search(r"typedef enum \{([^}]*)\}\s*" + name + r"\s*;", text).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"(LBM_\w+)\s*=\s*(\d+)", body)}


def test_binding_enums_match_the_header():
    """The ctypes binding passes enum values by number: they must be the header's."""
    kinds = _header_enum("lbm_kind")
    assert {("LBM_" + k.upper()): v for k, v in lbm.KINDS.items()} == kinds
    dtypes = _header_enum("lbm_dtype")
    assert {"LBM_" + k.upper(): v for k, v in lbm.DTYPES.items()} == dtypes
    assert {"LBM_" + k.upper(): v for k, v in lbm.EQS.items()} == _header_enum("lbm_eq")
    assert {"LBM_NCDE_" + k.upper(): v for k, v in lbm.NCDE_VARIANTS.items()} == _header_enum("lbm_ncde_variant")
    assert {"LBM_GATHER_" + k.upper(): v for k, v in lbm.GATHERS.items()} == _header_enum("lbm_gather")
    assert {v: k for k, v in _header_enum("lbm_status").items()} == lbm.STATUS
