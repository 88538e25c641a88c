"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and its host-side FC-Gram table builder agrees with the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fcsdnn.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2506_19370_gb300 import build, fcsdnn
    if not os.path.exists(fcsdnn.LIB_PATH):
        build.build()
    return fcsdnn.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("fc_setup", "fc_derivative", "sdnn_classify", "av_assemble", "euler_rhs", "rk_stage",
              "patch_exchange"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2506_19370_gb300 import fcsdnn
    names = declared_functions()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(fcsdnn.EXPORTS) == names


@pytest.mark.parametrize("d,C", [(5, 25), (2, 25), (5, 24), (5, 26), (5, 27), (5, 32), (5, 48)])
def test_table_builder_matches_oracle(lib, d, C):
    # the library builds its tables in double-double (Lagrange basis,
    # Householder QR); the oracle at 40 digits (Gram basis, mpmath QR)
    from oracle import fcgram
    from paper_2506_19370_gb300 import fcsdnn
    A_lib = fcsdnn.build_table(d, C)
    A_or, _ = fcgram.continuation_tables(d, C)
    scale = np.abs(A_or).max()
    assert np.abs(A_lib - A_or).max() <= 4e-16 * scale


def test_errors_are_reported(lib):
    from paper_2506_19370_gb300 import fcsdnn
    assert lib.fcs_strerror(-2) == b"fringe point without a donor outside the donor's own fringe"
    out = np.zeros(5, dtype=np.float64)
    assert lib.fcs_build_table(1, 25, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == -1
    h = ctypes.c_void_p()
    assert lib.fc_setup(ctypes.byref(h), 5, 25, None, 0, None) == -1
